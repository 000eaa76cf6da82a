// Pilot-wave sampler kernel for sm_103a.
//
// One group of threads (a warp, a named-barrier group inside a CTA, or a
// thread-block cluster when the frontier exceeds one CTA's shared memory) owns
// one Markov chain (Alg. 1 / Alg. 2) for its whole life: it walks every layer
// of the circuit, keeps the frontier tensor of the plan's sweep in shared
// memory, evaluates the candidate amplitudes amp(C_t, y) of each resampled
// qubit with the plan's program of fused passes, and draws the update from the
// normalised conditional with a counter-based Philox stream. Only the packed
// output bits (and the optional amplitude trace) reach HBM: the kernel is
// bound by latency (group barriers, dependent shared-memory and arithmetic
// chains of one chain) and FP32 arithmetic, not by DRAM.
//
// Per block of resampled qubits the group first builds every table the block
// needs (one parallel phase), then runs the fused passes back to back with one
// group barrier each, then reads out the block's conditional amplitudes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "dense.h"
#include "pw_internal.h"
#include "smem_layout.h"

namespace pw {

// --------------------------------------------------------------- complex
template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename R> __device__ __forceinline__ typename CT<R>::T mk(R re, R im) {
    typename CT<R>::T c;
    c.x = re;
    c.y = im;
    return c;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C c;
    c.x = a.x * b.x - a.y * b.y;
    c.y = a.x * b.y + a.y * b.x;
    return c;
}
// a*b + c
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {
    C r;
    r.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
    r.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
    return r;
}
__device__ __forceinline__ float scl(float v, int e) { return ldexpf(v, e); }
__device__ __forceinline__ double scl(double v, int e) { return ldexp(v, e); }
__device__ __forceinline__ float rmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double rmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float rabs(float a) { return fabsf(a); }
__device__ __forceinline__ double rabs(double a) { return fabs(a); }
__device__ __forceinline__ int rexp(float v) {
    int e;
    frexpf(v, &e);
    return e;
}
__device__ __forceinline__ int rexp(double v) {
    int e;
    frexp(v, &e);
    return e;
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): the two round multipliers and the two
// Weyl key increments of the published definition.
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Uniform in [0,1) with 53 random bits: top 27 bits of w0, top 26 of w1.
__device__ __forceinline__ double draw_u(uint64_t seed, uint64_t sample, uint32_t op_id, uint32_t purpose) {
    uint32_t c[4] = {(uint32_t)sample, (uint32_t)(sample >> 32), op_id, purpose};
    philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6)) * (1.0 / 9007199254740992.0);
}

// ----------------------------------------------------------- parameters
struct KParams {
    const unsigned char* blob;
    DevPlanOffsets off;
    DevPlanHeader hdr;
    SmemLayout sm;
    uint64_t seed, first, count;
    uint64_t* out_bits;
    double* trace;
    unsigned long long* counters;
    int tpc, gpc;
    int mode;           // MODE_SAMPLE or MODE_AMP
    const uint64_t* in_bits;
    double* amp_out;
    int amp_layer, amp_block, amp_pos;
    int cr;             // CTAs (one thread-block cluster) per chain; 1: one group per chain
    int wloc;           // log2 of the frontier entries held by one CTA when cr > 1
    // HBM engine (hdr.dense_mask != 0 or hbm = 1): the frontiers and the right
    // environments live in HBM; a launch runs every chain from yield point
    // y_from (-1: the start) to the next one, where it saves the chain state
    int hbm;
    int y_from;
    int ybase[8];                 // first yield point of layer m
    void* gL;                     // frontiers: chain c at gL + c * 2^(S P) entries (every layer)
    void* gR;                     // right environments: chain c at gR + c * strideR entries
    uint64_t strideR;
    unsigned char* gState;        // saved chain states, state_bytes each
    int state_off, state_bytes;   // the saved part of a group's shared memory
    void* gOps;                   // dense operators: pass i, chain c at (i * nch + c) * 2^(2k) entries
    void* gDiag;                  // epilogue tables: (i * nch + c) * 4 * 32 entries
    uint64_t nch;                 // chains the HBM buffers hold
};

enum { MODE_SAMPLE = 0, MODE_AMP = 1 };
enum { CNT_NEAR = 0, CNT_ZERO = 1, CNT_DENSE = 2 };   // CNT_DENSE: a bounded wait of a dense pass ran out

template <typename T> __device__ __forceinline__ const T* P_(const KParams& p, int64_t off) {
    return reinterpret_cast<const T*>(p.blob + off);
}

// The threads that run one phase of one chain: the whole group (named
// barrier over tpc threads), its first four warps (another named barrier;
// only when one group fills the CTA) or its first warp (warp barrier), the
// smaller ones for tensors too small to feed the group.
struct Grp {
    int lt, nt, gid, tpc;
    bool warp;
    bool clus;   // the phase spans the CTAs of a cluster (distributed frontier)
    __device__ __forceinline__ void sync() const {
        if (clus) {
            asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        } else if (warp || tpc == 32) {
            __syncwarp();
        } else if (nt < tpc) {
            // a subgroup of the first nt threads (whole warps) of a group that
            // fills its CTA: its own named barrier
            asm volatile("bar.sync %0, %1;" ::"r"(gid + 9), "r"(nt) : "memory");
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(gid + 1), "r"(tpc) : "memory");
        }
    }
};

// Per-chain view of the shared-memory group.
template <typename R> struct Chain {
    using C = typename CT<R>::T;
    C* L;         // frontier tensor, 2^W (top legs in the low S bits)
    C* Rt;        // right environments, K x 2^Wl
    int* Rexp;    // their power-of-two exponents
    C* rowdot;    // 2^S
    C* wt;        // readout slot weights: products over the low S/2 and the high S - S/2 slots
    C* T;         // 2^max_block
    C* sa;        // the current block's sites: mixer A'_m of site i at sa[4i .. 4i+3]
    int* sinfo;   // then their qubit, trace row and monomial flag, max_block each
    C* tab;       // tables of one block program
    DevStage* stg;    // stage descriptors of one block program
    double* ud;   // the chain's UpdateState draws, one per sampled gate
    float* uf;    // the same draws rounded to FP32 (fast path of the decision)
    C* part;      // partial sums, one per thread
    C* fslot;     // S x 2 per-slot readout factors
    R* red;       // 32 reduction scratch
    uint8_t* s;   // chain state s
    uint8_t* x;   // frame x (Alg. 2)
    uint8_t* xmix;    // frame during each one-qubit layer, [(P+1) n]
    uint8_t* gframe;  // frame bits of each diagonal gate at its time
    C* segfac;    // one-qubit diagonal factors per (qubit, segment), [n][P+1][2]
    int* misc;    // [0] exponent of L, [1] pending rescale, [2..17] role slots, [18..19] clean state
    // distributed frontier (cluster of p.cr CTAs per chain)
    int rank;            // this CTA's rank in the cluster (0 when cr == 1)
    C** rL;              // every rank's part of L (generic addresses, table in shared memory)
    double2* pd;         // this CTA's FP64 partial readout sums, 2^S
    float* cmax;         // this CTA's max |L|
};

// A chain is clean while every Kraus draw took operator 0 (misc[18] = 1):
// its frame is zero and its segment factors are the plan's fixed ones, so
// the host-evaluated variant tables hold for it.
enum { MISC_CLEAN = 18, MISC_DIRTY_EVENT = 19 };

template <typename R>
__device__ __forceinline__ bool chain_clean(const KParams& p, const Chain<R>& ch) {
    return !p.hdr.has_frame || (p.hdr.clean_tables && p.mode == MODE_SAMPLE && ch.misc[MISC_CLEAN] != 0);
}

// Frame-conjugated one-qubit gate A'_{m,q}[o][i] = A[o^x][i^x] (PropagateX).
template <typename R>
__device__ __forceinline__ typename CT<R>::T mixel(const KParams& p, const Chain<R>& ch, int m, int q, int o, int i) {
    const int xb = p.hdr.has_frame ? ch.xmix[m * p.hdr.n + q] : 0;
    const size_t base = ((size_t)m * p.hdr.n + q) * 8 + 2 * (((o ^ xb) << 1) | (i ^ xb));
    if constexpr (sizeof(R) == 4) {
        return *reinterpret_cast<const float2*>(P_<float>(p, p.off.mix_f) + base);
    } else {
        return *reinterpret_cast<const double2*>(P_<double>(p, p.off.mix_d) + base);
    }
}

// D'_g(a0 on q0, a1 on q1): a diagonal gate conjugated by the frame at its time.
template <typename R>
__device__ __forceinline__ typename CT<R>::T gatel(const KParams& p, const Chain<R>& ch, int g, int a0, int a1) {
    const DevCostGate* G = P_<DevCostGate>(p, p.off.cost_gates) + g;
    const int f = p.hdr.has_frame ? ch.gframe[g] : 0;
    const int idx = (a0 ^ (f & 1)) | ((a1 ^ ((f >> 1) & 1)) << 1);
    if constexpr (sizeof(R) == 4) {
        return *reinterpret_cast<const float2*>(G->f + 2 * idx);
    } else {
        return *reinterpret_cast<const double2*>(G->d + 2 * idx);
    }
}

// D'_g with qubit qa set to va and the other qubit of g set to vb.
template <typename R>
__device__ __forceinline__ typename CT<R>::T gate_pair(const KParams& p, const Chain<R>& ch, int g, int qa, int va, int vb) {
    const DevCostGate* G = P_<DevCostGate>(p, p.off.cost_gates) + g;
    return G->q0 == qa ? gatel<R>(p, ch, g, va, vb) : gatel<R>(p, ch, g, vb, va);
}

// Entry e of micro-op o's table (MAT1: e = out*2 + in; DIAG: its own bits).
template <typename R>
__device__ typename CT<R>::T build_entry(const KParams& p, const Chain<R>& ch, const DevMicroOp& o, int e) {
    using C = typename CT<R>::T;
    const int32_t* gref = P_<int32_t>(p, p.off.gate_refs);
    const C one = mk<R>(1, 0), zero = mk<R>(0, 0);
    switch (o.recipe) {
        case RC_EXPAND:
            return (e & 1) == 0 ? one : zero;
        case RC_SUMOUT1:
            return (e >> 1) == 0 ? one : zero;
        case RC_SUMOUT_MIX:
            return (e >> 1) == 0 ? mixel<R>(p, ch, o.layer, o.qa, ch.s[o.qa], e & 1) : zero;
        case RC_REPLACE: {
            const int aout = e >> 1, ain = e & 1;   // out: new site qb, in: eliminated site qa
            C v = o.layer >= 0 ? mixel<R>(p, ch, o.layer, o.qa, ch.s[o.qa], ain) : one;
            for (int i = 0; i < o.gcount; ++i) v = cmul(v, gate_pair<R>(p, ch, gref[o.glist + i], o.qa, ain, aout));
            return v;
        }
        case RC_BREPLACE: {
            const int aout = e >> 1, ain = e & 1;   // out: site qa, in: site qb
            C v = one;
            for (int i = 0; i < o.gcount; ++i) v = cmul(v, gate_pair<R>(p, ch, gref[o.glist + i], o.qa, aout, ain));
            return v;
        }
        case RC_EDGE: {
            const int a = e & 1, b = (e >> 1) & 1;
            C v = one;
            for (int i = 0; i < o.gcount; ++i) v = cmul(v, gate_pair<R>(p, ch, gref[o.glist + i], o.qa, a, b));
            return v;
        }
        case RC_SITE: {
            // Segments z^0..z^{layer-1} of qubit qa: the open ones are the low
            // bits of e, a fixed top takes the chain's bit. Value:
            // <z^0|A_0|0> prod_l A'_l[z^l][z^{l-1}] prod_l segfac(q, l)[z^l].
            const int q = o.qa, nseg = o.layer;
            int z[8];
            for (int l = 0; l < nseg; ++l) z[l] = (e >> l) & 1;
            if (o.fixed_top) z[nseg - 1] = ch.s[q];
            C v = mixel<R>(p, ch, 0, q, z[0], 0);
            for (int l = 1; l < nseg; ++l) v = cmul(v, mixel<R>(p, ch, l, q, z[l], z[l - 1]));
            if (p.hdr.has_segfac) {
                const int P1 = p.hdr.P + 1;
                for (int l = 0; l < nseg; ++l) v = cmul(v, ch.segfac[((size_t)q * P1 + l) * 2 + z[l]]);
            }
            return v;
        }
        case RC_CONST_EDGES: {
            C v = one;
            const DevCostGate* G = P_<DevCostGate>(p, p.off.cost_gates);
            for (int i = 0; i < o.gcount; ++i) {
                const int g = gref[o.glist + i];
                v = cmul(v, gatel<R>(p, ch, g, ch.s[G[g].q0], ch.s[G[g].q1]));
            }
            return v;
        }
    }
    return one;
}

// Tables and stage descriptors of one block program (stages [sb, sb + ns),
// ntab entries). Every entry is produced by one thread: precomputed stages
// select the variant of their dependency bits, the others are built from the
// chain's state. pend_exp (a power of two) is folded into the first stage;
// with exact = false the scalar-only factors (RC_CONST_EDGES), which change
// the amplitudes' overall scale but no conditional, are skipped.
template <typename R>
__device__ void build_tables(const KParams& p, const Chain<R>& ch, const Grp& g, int sb, int ns, int ntab,
                             int pend_exp, bool exact) {
    using C = typename CT<R>::T;
    const DevStage* ST = P_<DevStage>(p, p.off.stages) + sb;
    const DevMicroOp* ops = P_<DevMicroOp>(p, p.off.micro);
    const bool clean = chain_clean<R>(p, ch);
    for (int i = g.lt; i < ns; i += g.nt) ch.stg[i] = ST[i];
    const Grp gl{g.lt, g.nt, g.gid, g.tpc, g.warp, false};
    gl.sync();   // the lookups below read this CTA's shared copy
    const DevStage* SS = ch.stg;
    for (int ef = g.lt; ef < ntab; ef += g.nt) {
        int si = 0;   // last stage with tab_off <= ef (offsets ascend)
        for (int hi = ns - 1; si < hi;) {
            const int mid = (si + hi + 1) >> 1;
            if (SS[mid].tab_off <= ef)
                si = mid;
            else
                hi = mid - 1;
        }
        const DevStage st = SS[si];
        const int e = ef - st.tab_off;
        C v;
        if (st.ndep != 0xFF && clean) {   // precomputed variant
            int var = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)   // (compile-time indices: the copy stays in registers)
                if (j < st.ndep) var |= ch.s[st.dep[j]] << j;
            const int size = st.type == ST_MAT ? 4 : (1 << st.arg);
            const size_t at = (size_t)st.var_off + (size_t)var * size + e;
            if constexpr (sizeof(R) == 4) {
                v = *reinterpret_cast<const float2*>(P_<float>(p, p.off.vtab_f) + 2 * at);
            } else {
                v = *reinterpret_cast<const double2*>(P_<double>(p, p.off.vtab_d) + 2 * at);
            }
        } else if (st.type == ST_MAT) {
            v = build_entry<R>(p, ch, ops[st.op_begin], e);
        } else {
            v = mk<R>(1, 0);
            for (int k = st.op_begin; k < st.op_end; ++k) {
                const DevMicroOp o = ops[k];
                if (!exact && o.recipe == RC_CONST_EDGES) continue;
                int loc = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < o.nbits) loc |= ((e >> o.fpos[j]) & 1) << j;
                v = cmul(v, build_entry<R>(p, ch, o, loc));
            }
        }
        if (exact && clean && si == 0) {
            // scale factors left out of the precomputed tables of this
            // program (the stages built here include their own)
            for (int s2 = 0; s2 < ns; ++s2) {
                if (SS[s2].ndep == 0xFF) continue;
                for (int k = SS[s2].op_begin; k < SS[s2].op_end; ++k)
                    if (ops[k].recipe == RC_CONST_EDGES) v = cmul(v, build_entry<R>(p, ch, ops[k], 0));
            }
        }
        if (si == 0 && pend_exp != 0) {
            v.x = scl(v.x, pend_exp);
            v.y = scl(v.y, pend_exp);
        }
        ch.tab[ef] = v;
    }
}

// (x[e], x[e | 1<<K]) <- M (x[e], x[e | 1<<K]) for every e with bit K clear.
// (The tiled pass treats every shape of M as general: branching on the shape
// inside the unrolled tile code made it spill and ran slower.)
template <typename C, int T, int K>
__device__ __forceinline__ void mat_stage(C (&x)[1 << T], C m00, C m01, C m10, C m11) {
#pragma unroll
    for (int e = 0; e < (1 << T); ++e) {
        if (e & (1 << K)) continue;
        const C x0 = x[e], x1 = x[e | (1 << K)];
        x[e] = cfma(m00, x0, cmul(m01, x1));
        x[e | (1 << K)] = cfma(m10, x0, cmul(m11, x1));
    }
}
// Shared-memory position of frontier / environment entry i: bits 4..7 of i
// are XORed into bits 0..3, so that warps striding over low index bits (a
// pass whose tile bits include them) spread over the banks. A bijection on
// [0, 2^W) for every W; entry 0 stays at position 0.
__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 4) & 15); }

// Frontier access: a CTA's own shared memory, or the parts held by the CTAs of
// a cluster (entry idx in rank idx >> wloc at offset idx & (2^wloc - 1)).
template <typename C> struct LocalAcc {
    C* buf;
    int base = 0;   // first entry held in buf (a cluster rank's part: rank << wloc)
    __device__ __forceinline__ C& operator()(int idx) const { return buf[swz(idx) - base]; }
    // entry b0 | o given swz(b0) and swz(o) (swz is linear over XOR, and b0
    // and o have no common bit; it leaves bits above 7 alone, so subtracting
    // a base of whole 256-entry multiples commutes with it)
    __device__ __forceinline__ C& at(int b0, int sb0, int o, int so) const { return buf[(sb0 ^ so) - base]; }
};
template <typename C> struct DistAcc {
    C* const* rl;   // every rank's part (a table in shared memory)
    C* loc;         // this CTA's part
    int wloc, rank;
    __device__ __forceinline__ C& operator()(int idx) const {
        const int r = idx >> wloc, o = swz(idx & ((1 << wloc) - 1));
        return r == rank ? loc[o] : rl[r][o];
    }
    __device__ __forceinline__ C& at(int b0, int sb0, int o, int so) const { return (*this)(b0 | o); }
};

// One tiled pass over tiles [t0, t1) of a 2^W-entry frontier by the threads of
// g: each thread loads tiles of 2^T entries (the pass's tile bits varying),
// runs the pass's stages on them in registers and stores them back.
template <typename R, int T, typename Acc>
__device__ void tile_pass(const KParams& p, const Chain<R>& ch, const Grp& g, const DevFused& f, int sb,
                          const Acc& acc, int t_begin, int t_end) {
    using C = typename CT<R>::T;
    constexpr int E = 1 << T;
    int msk[4] = {0, 0, 0, 0}, smk[4] = {0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < T; ++k) {
        msk[k] = 1 << f.tbits[k];
        smk[k] = swz(msk[k]);
    }
    int sb4[4] = {f.tbits[0], f.tbits[1], f.tbits[2], f.tbits[3]};
#pragma unroll
    for (int a = 1; a < T; ++a)
#pragma unroll
        for (int b = a; b > 0; --b)
            if (sb4[b] < sb4[b - 1]) {
                const int t = sb4[b];
                sb4[b] = sb4[b - 1];
                sb4[b - 1] = t;
            }
    const DevStage* stg = ch.stg + sb;
    for (int t0 = t_begin + g.lt; t0 < t_end; t0 += g.nt) {
        int b0 = t0;
#pragma unroll
        for (int k = 0; k < T; ++k) b0 = ((b0 >> sb4[k]) << (sb4[k] + 1)) | (b0 & ((1 << sb4[k]) - 1));
        const int sb0 = swz(b0);
        C x[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int o = 0, so = 0;
#pragma unroll
            for (int k = 0; k < T; ++k)
                if (e & (1 << k)) {
                    o |= msk[k];
                    so ^= smk[k];
                }
            x[e] = acc.at(b0, sb0, o, so);
        }
        for (int s = 0; s < f.nst; ++s) {
            const uint8_t type = stg[s].type, arg = stg[s].arg;
            const C* tab = ch.tab + stg[s].tab_off;
            if (type == ST_MAT) {
                const C m00 = tab[0], m01 = tab[1], m10 = tab[2], m11 = tab[3];
                if constexpr (T >= 1) {
                    switch (arg) {
                        case 0: mat_stage<C, T, 0>(x, m00, m01, m10, m11); break;
                        case 1: if constexpr (T >= 2) mat_stage<C, T, (T >= 2 ? 1 : 0)>(x, m00, m01, m10, m11); break;
                        case 2: if constexpr (T >= 3) mat_stage<C, T, (T >= 3 ? 2 : 0)>(x, m00, m01, m10, m11); break;
                        default: if constexpr (T >= 4) mat_stage<C, T, (T >= 4 ? 3 : 0)>(x, m00, m01, m10, m11); break;
                    }
                }
            } else {
                int tb0 = 0;
                int db[5];
#pragma unroll
                for (int j = 0; j < 5; ++j) db[j] = stg[s].dbits[j];
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (j < arg) tb0 |= ((b0 >> db[j]) & 1) << j;
                int pm[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) pm[k] = stg[s].tpos[k] != 0xFF ? 1 << stg[s].tpos[k] : 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int t = 0;
#pragma unroll
                    for (int k = 0; k < T; ++k)
                        if (e & (1 << k)) t |= pm[k];
                    x[e] = cmul(x[e], tab[tb0 | t]);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            int o = 0, so = 0;
#pragma unroll
            for (int k = 0; k < T; ++k)
                if (e & (1 << k)) {
                    o |= msk[k];
                    so ^= smk[k];
                }
            acc.at(b0, sb0, o, so) = x[e];
        }
    }
}

// A pass on a tensor with fewer tiles than threads: its stages run one after
// another over the whole tensor (a pair per thread for a matrix, an entry per
// thread for a diagonal), with a barrier between stages. Each stage's fields
// are read into registers once (the element loop stores to shared memory, so
// they would otherwise be reloaded for every element).
template <typename R>
__device__ void flat_pass(const KParams& p, const Chain<R>& ch, const Grp& g, const DevFused& f, int sb,
                          typename CT<R>::T* buf, int W) {
    using C = typename CT<R>::T;
    const int N = 1 << W;
    const DevStage* stg = ch.stg + sb;
    for (int s = 0; s < f.nst; ++s) {
        const uint8_t type = stg[s].type, arg = stg[s].arg;
        const C* tab = ch.tab + stg[s].tab_off;
        if (type == ST_MAT) {
            const int bt = arg == 0 ? f.tbits[0] : arg == 1 ? f.tbits[1] : arg == 2 ? f.tbits[2] : f.tbits[3];
            const uint8_t form = stg[s].form;
            const C m00 = tab[0], m01 = tab[1], m10 = tab[2], m11 = tab[3];
            for (int pi = g.lt; pi < (N >> 1); pi += g.nt) {
                const int i0 = ((pi >> bt) << (bt + 1)) | (pi & ((1 << bt) - 1));
                const int i1 = swz(i0 | (1 << bt)), j0 = swz(i0);
                const C x0 = buf[j0];
                if (form == MF_EXPAND) {
                    // a copy; the first stage of a block program also carries the
                    // pending power of two and, in exact mode, the scale-only
                    // factors of the program (any complex value), so it multiplies
                    const C y = sb + s == 0 ? cmul(m00, x0) : x0;
                    buf[j0] = y;
                    buf[i1] = y;
                } else if (form == MF_ROW0) {
                    buf[j0] = cfma(m00, x0, cmul(m01, buf[i1]));
                    buf[i1] = mk<R>(0, 0);
                } else {
                    const C x1 = buf[i1];
                    buf[j0] = cfma(m00, x0, cmul(m01, x1));
                    buf[i1] = cfma(m10, x0, cmul(m11, x1));
                }
            }
        } else {
            int db[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) db[j] = stg[s].dbits[j];
            for (int idx = g.lt; idx < N; idx += g.nt) {
                int t = 0;
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (j < arg) t |= ((idx >> db[j]) & 1) << j;
                buf[swz(idx)] = cmul(buf[swz(idx)], tab[t]);
            }
        }
        if (s + 1 < f.nst) g.sync();
    }
}

template <typename R, int T>
__device__ __forceinline__ void tile_pass_any(const KParams& p, const Chain<R>& ch, const Grp& g, const DevFused& f,
                                              int sb, typename CT<R>::T* buf, int W, bool dist) {
    using C = typename CT<R>::T;
    const int ntiles = (1 << W) >> T;
    bool crosses = false;   // split frontier, a tile bit among the rank bits: tiles span CTAs
    if (dist)
        for (int k = 0; k < T; ++k) crosses |= f.tbits[k] >= p.wloc;
    if (crosses) {
        // rank r takes the tiles whose number has r in its top bits
        const int per = ntiles / p.cr;
        tile_pass<R, T>(p, ch, g, f, sb, DistAcc<C>{ch.rL, ch.L, p.wloc, ch.rank}, ch.rank * per, (ch.rank + 1) * per);
    } else if (!dist && ntiles < g.nt) {
        flat_pass<R>(p, ch, g, f, sb, buf, W);
    } else {
        // this CTA's own entries: the whole tensor, or (split frontier, tile
        // bits below the rank bits) the tiles of this rank's part
        const int per = dist ? ntiles / p.cr : ntiles;
        const int t0 = dist ? ch.rank * per : 0;
        tile_pass<R, T>(p, ch, g, f, sb, LocalAcc<C>{dist ? ch.L : buf, dist ? ch.rank << p.wloc : 0}, t0, t0 + per);
    }
}

// Run passes [fb, fe) (their stages start at stage sb0 of the block) on buf.
template <typename R>
__device__ void run_passes(const KParams& p, const Chain<R>& ch, const Grp& g, int fb, int fe, int sb0,
                           typename CT<R>::T* buf, int W, bool dist = false) {
    const DevFused* F = P_<DevFused>(p, p.off.fused);
    if (fb >= fe) return;
    DevFused fnext = F[fb];
    for (int fi = fb; fi < fe; ++fi) {
        const DevFused f = fnext;
        if (fi + 1 < fe) fnext = F[fi + 1];   // in flight during this pass
        const int sb = f.st_begin - sb0;
        switch (f.ntb) {
            case 0: tile_pass_any<R, 0>(p, ch, g, f, sb, buf, W, dist); break;
            case 1: tile_pass_any<R, 1>(p, ch, g, f, sb, buf, W, dist); break;
            case 2: tile_pass_any<R, 2>(p, ch, g, f, sb, buf, W, dist); break;
            case 3: tile_pass_any<R, 3>(p, ch, g, f, sb, buf, W, dist); break;
            default: tile_pass_any<R, 4>(p, ch, g, f, sb, buf, W, dist); break;
        }
        g.sync();
    }
}

// Max over the threads of g of a per-thread value (broadcast).
template <typename R>
__device__ R group_max(const Chain<R>& ch, const Grp& g, R v) {
    for (int o = 16; o > 0; o >>= 1) v = rmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (g.warp || g.nt <= 32) return v;
    const int nw = (g.nt + 31) >> 5;
    if ((g.lt & 31) == 0) ch.red[g.lt >> 5] = v;
    g.sync();
    R m = ch.red[0];
    for (int w = 1; w < nw; ++w) m = rmax(m, ch.red[w]);
    g.sync();
    return m;
}

// Exponent e with 2^-e * mx in [0.5, 1); 0 for zero or non-finite mx.
template <typename R> __device__ __forceinline__ int scale_exp(R mx) {
    if (!(mx > (R)0) || !isfinite(mx)) return 0;
    return rexp(mx);
}

// Kraus draw of Eq. (5) at the true bits s XOR x: the smallest i with
// u * total < cum[cb][i] (same rule as UpdateState). Draws within 1e-6 of a
// boundary are counted when count_near is set.
template <typename R>
__device__ __forceinline__ int kraus_pick(const KParams& p, const Chain<R>& ch, const DevChannel& c, const double* cum,
                                          uint64_t sample_id, bool count_near) {
    int cb = 0;
    for (int i = 0; i < c.nq; ++i) cb |= (ch.s[c.q[i]] ^ ch.x[c.q[i]]) << i;
    const double* row = cum + c.cum_off + (size_t)cb * c.k;
    const double total = row[c.k - 1];
    const double u = draw_u(p.seed, sample_id, (uint32_t)c.op_id, 1u);
    int pick = c.k - 1;
    for (int i = 0; i < c.k; ++i)
        if (u * total < row[i]) {
            pick = i;
            break;
        }
    if (count_near)
        for (int i = 0; i + 1 < c.k; ++i)
            if (fabs(u * total - row[i]) < 1e-6 * total) {
                if (ch.rank == 0) atomicAdd(&p.counters[CNT_NEAR], 1ull);
                break;
            }
    return pick;
}

// The drawn Kraus operator, then Alg. 2: every anti-diagonal factor flips
// x[q] and becomes the diagonal M sigma_X; each diagonal factor is conjugated
// by the (updated) frame and multiplied into the qubit's current segment.
template <typename R>
__device__ void apply_channel(const KParams& p, const Chain<R>& ch, const DevChannel& c, const double* cum,
                              const DevKrausFactor* fac, uint64_t sample_id, int seg, bool count_near) {
    using C = typename CT<R>::T;
    const int pick = kraus_pick<R>(p, ch, c, cum, sample_id, count_near);
    const int P1 = p.hdr.P + 1;
    for (int f = 0; f < c.nq; ++f) {
        const DevKrausFactor F = fac[c.fac_off + pick * c.nq + f];
        if (F.antidiag) ch.x[F.q] ^= 1;
        C d0 = mk<R>((R)F.d[0], (R)F.d[1]), d1 = mk<R>((R)F.d[2], (R)F.d[3]);
        if (ch.x[F.q]) {
            const C t = d0;
            d0 = d1;
            d1 = t;
        }
        C* sf = ch.segfac + ((size_t)F.q * P1 + seg) * 2;
        sf[0] = cmul(sf[0], d0);
        sf[1] = cmul(sf[1], d1);
    }
}

// Per-slot readout factors of block k: cross edges of the top segment to
// unabsorbed qubits (at their current bits) and, for sites resampled in an
// earlier block, their mixer weight A'_m[s][top]. Also records which slot
// holds the i-th site of the block.
template <typename R>
__device__ void build_fslot(const KParams& p, const Chain<R>& ch, const Grp& g, int m, const DevBlockRange& br) {
    using C = typename CT<R>::T;
    const DevLiveSlot* live = P_<DevLiveSlot>(p, p.off.live_slots) + br.live_begin;
    const int32_t* gref = P_<int32_t>(p, p.off.gate_refs);
    const DevCostGate* G = P_<DevCostGate>(p, p.off.cost_gates);
    const bool clean = chain_clean<R>(p, ch);
    // (slots and sites start on other threads than the table entries of
    // build_tables, so that their global-memory loads overlap)
    const int lts = g.nt >= 64 ? (g.lt + g.nt / 2) % g.nt : g.lt;
    const int lti = g.nt >= 64 ? (g.lt + 3 * g.nt / 4) % g.nt : g.lt;
    for (int j = lts; j < p.hdr.S; j += g.nt) {
        const DevLiveSlot sl = live[j];
        if (sl.q >= 0 && sl.role >= 0) ch.misc[2 + sl.role] = j;
        if (sl.ndep != 0xFF && clean) {
            int var = 0;
            for (int d = 0; d < sl.ndep; ++d) var |= ch.s[sl.dep[d]] << d;
            const size_t at = (size_t)sl.var_off + 2 * (size_t)var;
            if constexpr (sizeof(R) == 4) {
                // 8-byte loads: variant tables start at any complex entry
                const float2* v = reinterpret_cast<const float2*>(P_<float>(p, p.off.vtab_f) + 2 * at);
                ch.fslot[2 * j] = v[0];
                ch.fslot[2 * j + 1] = v[1];
            } else {
                const double* d = P_<double>(p, p.off.vtab_d) + 2 * at;
                ch.fslot[2 * j] = mk<R>(d[0], d[1]);
                ch.fslot[2 * j + 1] = mk<R>(d[2], d[3]);
            }
            continue;
        }
        C f0 = mk<R>(1, 0), f1 = mk<R>(0, 0);
        if (sl.q >= 0) {
            f1 = mk<R>(1, 0);
            for (int i = 0; i < sl.dcount; ++i) {
                const int gg = gref[sl.dlist + i];
                const int w = G[gg].q0 == sl.q ? G[gg].q1 : G[gg].q0;
                f0 = cmul(f0, gate_pair<R>(p, ch, gg, sl.q, 0, ch.s[w]));
                f1 = cmul(f1, gate_pair<R>(p, ch, gg, sl.q, 1, ch.s[w]));
            }
            if (sl.role < 0) {
                f0 = cmul(f0, mixel<R>(p, ch, m, sl.q, ch.s[sl.q], 0));
                f1 = cmul(f1, mixel<R>(p, ch, m, sl.q, ch.s[sl.q], 1));
            } else {
                ch.misc[2 + sl.role] = j;
            }
        }
        ch.fslot[2 * j] = f0;
        ch.fslot[2 * j + 1] = f1;
    }
    // the block's sites for the resampling warp (loaded here, ahead of the
    // passes, so that their global-memory latency is off its path)
    const DevBlockSite* sites = P_<DevBlockSite>(p, p.off.block_sites) + br.site_begin;
    const int nb = br.site_end - br.site_begin, mb = p.hdr.max_block;
    for (int i = lti; i < nb; i += g.nt) {
        const DevBlockSite st = sites[i];
        ch.sa[4 * i] = mixel<R>(p, ch, m, st.q, 0, 0);
        ch.sa[4 * i + 1] = mixel<R>(p, ch, m, st.q, 0, 1);
        ch.sa[4 * i + 2] = mixel<R>(p, ch, m, st.q, 1, 0);
        ch.sa[4 * i + 3] = mixel<R>(p, ch, m, st.q, 1, 1);
        ch.sinfo[i] = st.q;
        ch.sinfo[mb + i] = st.trace_row;
        ch.sinfo[2 * mb + i] = st.monomial;
    }
}

// Readout of block k of layer m. The frontier index is top legs (low S bits)
// + lower legs (high bits): T(tops of the block's sites) =
// sum_{l,h} L[l, h] R_k[l] prod_slots fslot[j][h_j], then the block's sites
// are resampled one after another (UpdateState of Alg. 1), contracting each
// resampled top with A'_m[s_new][.] before moving to the next site.
template <typename R>
__device__ void readout_and_sample(const KParams& p, const Chain<R>& ch, const Grp& g, int m, int k,
                                   const DevBlockRange& br, uint64_t chain, bool dist = false) {
    using C = typename CT<R>::T;
    const DevPlanHeader& h = p.hdr;
    const int S = h.S, Wl = S * (m - 1);
    const int NL = 1 << Wl, H = 1 << S;
    const C zero = mk<R>(0, 0), one = mk<R>(1, 0);
    const C* Rk = ch.Rt + (size_t)k * NL;
    const C* L = ch.L;

    // 1) rowdot[h] = sum_l L[l*H + h] R_k[l] (coalesced), and max |L|. With a
    //    distributed frontier every CTA sums its own rows l (its share of the
    //    lower legs); the partial sums are then added across the cluster in
    //    FP64, in rank order, identically in every CTA.
    //    With a single row (layer 1, one CTA) there is nothing to sum: the
    //    collapse below reads L directly and finds max |L| on the way.
    const bool direct = NL == 1 && !dist;
    R mx = 0;
    const int NLl = dist ? NL / p.cr : NL;    // rows held by this CTA
    const int l0 = dist ? ch.rank * NLl : 0;  // first of them
    if (direct) {
    } else if (g.nt >= H) {
        const int hh = g.lt & (H - 1), step = g.nt / H;
        C acc[4] = {zero, zero, zero, zero};   // independent chains for latency
        int l = g.lt / H;
        for (; l + 3 * step < NLl; l += 4 * step) {
            C v[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) v[a] = L[swz((l + a * step) * H + hh)];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                acc[a] = cfma(v[a], Rk[swz(l0 + l + a * step)], acc[a]);
                mx = rmax(mx, rmax(rabs(v[a].x), rabs(v[a].y)));
            }
        }
        for (; l < NLl; l += step) {
            const C v = L[swz(l * H + hh)];
            acc[0] = cfma(v, Rk[swz(l0 + l)], acc[0]);
            mx = rmax(mx, rmax(rabs(v.x), rabs(v.y)));
        }
        ch.part[g.lt] = mk<R>(acc[0].x + acc[1].x + acc[2].x + acc[3].x, acc[0].y + acc[1].y + acc[2].y + acc[3].y);
    } else {
        // eight rows in flight per thread (the frontier of the HBM engine is
        // read from HBM here), summed in a fixed order
        for (int hh = g.lt; hh < H; hh += g.nt) {
            C acc[8] = {zero, zero, zero, zero, zero, zero, zero, zero};
            int l = 0;
            for (; l + 8 <= NLl; l += 8) {
                C v[8];
#pragma unroll
                for (int a = 0; a < 8; ++a) v[a] = L[swz((l + a) * H + hh)];
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    acc[a] = cfma(v[a], Rk[swz(l0 + l + a)], acc[a]);
                    mx = rmax(mx, rmax(rabs(v[a].x), rabs(v[a].y)));
                }
            }
            for (; l < NLl; ++l) {
                const C v = L[swz(l * H + hh)];
                acc[0] = cfma(v, Rk[swz(l0 + l)], acc[0]);
                mx = rmax(mx, rmax(rabs(v.x), rabs(v.y)));
            }
#pragma unroll
            for (int a = 1; a < 8; ++a) {
                acc[0].x += acc[a].x;
                acc[0].y += acc[a].y;
            }
            ch.rowdot[hh] = acc[0];
        }
    }
    // The readout weight of a top configuration hv is the product over the S
    // slots of fslot[slot][bit]; it factorises into a product over the low S/2
    // slots and one over the rest, tabulated here (fslot is final since the
    // block's passes began).
    const int Sa = S >> 1, Na = 1 << Sa, Nw = Na + (1 << (S - Sa));
    for (int e = g.lt; e < Nw; e += g.nt) {
        const bool lo = e < Na;
        const int v = lo ? e : e - Na, j0 = lo ? 0 : Sa, j1 = lo ? Sa : S;
        C w = one;
        for (int j = j0; j < j1; ++j) w = cmul(w, ch.fslot[2 * j + ((v >> (j - j0)) & 1)]);
        ch.wt[e] = w;
    }
    const Grp gl{g.lt, g.nt, g.gid, g.tpc, g.warp, false};   // this CTA only
    if (!direct) mx = group_max<R>(ch, gl, mx);
    gl.sync();
    if (!direct && g.nt >= H && g.lt < H) {
        C acc = zero;
        for (int j = g.lt; j < g.nt; j += H) {
            acc.x += ch.part[j].x;
            acc.y += ch.part[j].y;
        }
        ch.rowdot[g.lt] = acc;
    }
    if (dist) {
        gl.sync();
        for (int hh = g.lt; hh < H; hh += g.nt) ch.pd[hh] = make_double2((double)ch.rowdot[hh].x, (double)ch.rowdot[hh].y);
        if (g.lt == 0) ch.cmax[0] = (float)mx;
        g.sync();   // cluster: every partial written
        for (int hh = g.lt; hh < H; hh += g.nt) {
            double sx = 0.0, sy = 0.0;
            for (int r = 0; r < p.cr; ++r) {
                const double2 v = static_cast<const double2*>(__cluster_map_shared_rank(ch.pd, r))[hh];
                sx += v.x;
                sy += v.y;
            }
            ch.rowdot[hh] = mk<R>((R)sx, (R)sy);
        }
        for (int r = 0; r < p.cr; ++r)
            mx = rmax(mx, (R) static_cast<const float*>(__cluster_map_shared_rank(ch.cmax, r))[0]);
        g.sync();   // cluster: partials consumed before anyone overwrites them
    }
    const int eL = ch.misc[0];
    const int escale = eL + ch.Rexp[k] + h.amp_exp;
    const bool target_block = p.mode == MODE_AMP && m == p.amp_layer && k == p.amp_block;
    if (!direct) {
        g.sync();
        if (g.lt == 0) {
            const int e = scale_exp<R>(mx);
            ch.misc[1] = -e;
            ch.misc[0] = eL + e;
        }
        if (p.mode == MODE_AMP && !target_block) {
            g.sync();
            return;
        }
    }

    // 2) collapse onto the block's tops: T[t] = sum over the other top slots
    //    of rowdot[hv] times the weight of hv, bit i of t = top of block site i.
    //    Work item u = (bin t, chunk c): the chunk fixes the lowest cb of the
    //    other slots' bits and enumerates the rest (subset walk of mask mh).
    //    With several chunks per bin the partials go to part[] and the
    //    resampling warp adds them in chunk order.
    const int nb = br.site_end - br.site_begin;
    const int NT = 1 << nb;
    int cb = 31 - __clz(g.nt) - nb;
    cb = cb < 0 ? 0 : (cb > S - nb ? S - nb : cb);
    const int ncb = 1 << cb;
    {
        int mh = ~br.rmask & (H - 1), mc = 0;
        for (int b = 0; b < cb; ++b) {
            const int low = mh & -mh;
            mc |= low;
            mh ^= low;
        }
        for (int u = g.lt; u < NT * ncb; u += g.nt) {
            const int t = u & (NT - 1), c = u >> nb;
            int base = 0;
            for (int i = 0; i < nb; ++i) base |= ((t >> i) & 1) << br.rslot[i];
            for (int b = 0, mm = mc; b < cb; ++b) {
                const int low = mm & -mm;
                if ((c >> b) & 1) base |= low;
                mm ^= low;
            }
            C acc = zero;
            int xh = 0;
            do {
                const int hv = base | xh;
                C v;
                if (direct) {
                    v = L[swz(hv)];
                    mx = rmax(mx, rmax(rabs(v.x), rabs(v.y)));
                } else {
                    v = ch.rowdot[hv];
                }
                acc = cfma(v, cmul(ch.wt[hv & (Na - 1)], ch.wt[Na + (hv >> Sa)]), acc);
                xh = (xh - mh) & mh;
            } while (xh != 0);
            if (direct) acc = cmul(acc, Rk[0]);
            if (ncb == 1)
                ch.T[t] = acc;
            else
                ch.part[u] = acc;
        }
    }
    if (direct) {
        // every entry of L was read by exactly one work item
        mx = group_max<R>(ch, gl, mx);
        g.sync();
        if (g.lt == 0) {
            const int e = scale_exp<R>(mx);
            ch.misc[1] = -e;
            ch.misc[0] = eL + e;
        }
        if (p.mode == MODE_AMP && !target_block) {
            g.sync();
            return;
        }
    }
    g.sync();

    // 3) sequential resampling of the block's sites by the first warp (their
    //    mixers and descriptors were staged in shared memory by build_fslot):
    //    each decision (FP64 conditional, the chain's precomputed Philox draw)
    //    is taken by every lane alike; the lanes then contract the resampled
    //    top away in parallel. The block's bits live in a register mask until they
    //    are written back.
    const int wsz = g.nt < 32 ? g.nt : 32;
    if (g.lt < wsz) {
        const int lane = g.lt;
        if (ncb > 1) {
            for (int t = lane; t < NT; t += wsz) {
                C a = ch.part[t];
                for (int c = 1; c < ncb; ++c) {
                    a.x += ch.part[t + c * NT].x;
                    a.y += ch.part[t + c * NT].y;
                }
                ch.T[t] = a;
            }
            __syncwarp();
        }
        const C* sa = ch.sa;   // staged by build_fslot
        const int* sq = ch.sinfo;
        const int* srow = sq + h.max_block;
        const int* smono = srow + h.max_block;
        unsigned sbits = 0;
        for (int i = 0; i < nb; ++i) sbits |= (unsigned)ch.s[sq[i]] << i;
        C* cur = ch.T;
        int size = 1 << nb;
        for (int i = 0; i < nb; ++i) {
            const C A00 = sa[4 * i], A01 = sa[4 * i + 1], A10 = sa[4 * i + 2], A11 = sa[4 * i + 3];
            const int sold = (sbits >> i) & 1;
            int snew = sold;
            bool stop = false;
            // every lane takes the same decision from the same (broadcast)
            // reads; only lane 0 writes outputs and counters
            {
                const bool w = lane == 0;
                const int row = srow[i], mono = smono[i];
                const int rest = (int)((sbits >> (i + 1)) << 1);   // later sites keep their bits
                const C c0 = cur[rest], c1 = cur[rest | 1];
                const C amp0 = cfma(A00, c0, cmul(A01, c1));
                const C amp1 = cfma(A10, c0, cmul(A11, c1));
                if (p.mode == MODE_AMP) {
                    if (i == p.amp_pos) {
                        const C a = sold ? amp1 : amp0;
                        if (w && ch.rank == 0) {
                            p.amp_out[2 * chain] = ldexp((double)a.x, escale);
                            p.amp_out[2 * chain + 1] = ldexp((double)a.y, escale);
                        }
                        stop = true;
                    }
                } else if (mono) {
                    // deterministic move: the nonzero of column s[q] of A'_m
                    const C a0 = sold ? A01 : A00;
                    snew = (a0.x != (R)0 || a0.y != (R)0) ? 0 : 1;
                } else {
                    if (w && p.trace && ch.rank == 0) {
                        double* tr = p.trace + ((size_t)chain * h.n_sampled + row) * 4;
                        tr[0] = ldexp((double)amp0.x, escale);
                        tr[1] = ldexp((double)amp0.y, escale);
                        tr[2] = ldexp((double)amp1.x, escale);
                        tr[3] = ldexp((double)amp1.y, escale);
                    }
                    // The draw is decided in FP64: u*P < p0 with p_y = |amp_y|^2.
                    // When the FP32 evaluation of the same quantities is farther
                    // than 4e-6 P from the boundary (its error is below 1e-6 P)
                    // it gives the same answer, and no FP64 work is needed.
                    const float f0 = fmaf((float)amp0.x, (float)amp0.x, (float)amp0.y * (float)amp0.y);
                    const float f1 = fmaf((float)amp1.x, (float)amp1.x, (float)amp1.y * (float)amp1.y);
                    const float fP = f0 + f1;
                    const float fd = fmaf(ch.uf[row], fP, -f0);
                    if (fP > 0.0f && isfinite(fP) && fabsf(fd) > 4e-6f * fP) {
                        snew = fd < 0.0f ? 0 : 1;
                    } else {
                        const double a0r = amp0.x, a0i = amp0.y, a1r = amp1.x, a1i = amp1.y;
                        const double p0 = fma(a0r, a0r, a0i * a0i), p1 = fma(a1r, a1r, a1i * a1i);
                        const double Pt = p0 + p1;
                        if (Pt > 0.0) {
                            const double up = ch.ud[row] * Pt;
                            snew = up < p0 ? 0 : 1;
                            if (w && fabs(up - p0) < 1e-6 * Pt && ch.rank == 0) atomicAdd(&p.counters[CNT_NEAR], 1ull);
                        } else if (w && ch.rank == 0) {
                            atomicAdd(&p.counters[CNT_ZERO], 1ull);   // zero-mass block: stay (Sec. 2)
                        }
                    }
                }
            }
            if (stop) break;
            sbits = (sbits & ~(1u << i)) | ((unsigned)snew << i);
            if (i + 1 == nb) break;   // (nothing reads the last contraction)
            // contract this site's top with its mixer weight at the new bit
            // (ping-pong between the two halves of the T area)
            const C w0 = snew ? A10 : A00, w1 = snew ? A11 : A01;
            size >>= 1;
            C* nxt = cur == ch.T ? ch.T + (1 << h.max_block) : ch.T;
            for (int r = lane; r < size; r += wsz) nxt[r] = cfma(w0, cur[2 * r], cmul(w1, cur[2 * r + 1]));
            cur = nxt;
            __syncwarp();
        }
        if (p.mode == MODE_SAMPLE)
            for (int i = lane; i < nb; i += wsz) ch.s[sq[i]] = (uint8_t)((sbits >> i) & 1);
    }
    g.sync();
}

// Cost section m (1..P+1), one wave after the other: the frame bits of the
// diagonal gates at their time, the one-qubit diagonal factors of segment m-1
// and the Kraus draws of the channels (Eq. 5; the channels after the last
// layer act on segment P). The items of a wave touch disjoint qubits and run
// in parallel over the group.
//
// A clean chain first draws every channel of the section at once: with a zero
// frame a draw depends only on s, so the order does not matter. If all draws
// give operator 0 the chain stays clean and nothing else changes (its gate
// frame bits stay zero and its segment factors are the fixed ones). Otherwise
// it becomes dirty: it takes the fixed factors of the earlier segments and
// runs the section wave by wave, which redraws the same counters in order.
template <typename R>
__device__ void cost_section(const KParams& p, const Chain<R>& ch, const Grp& G, int m, uint64_t sample_id) {
    using C = typename CT<R>::T;
    const int P1 = p.hdr.P + 1;
    const int32_t* cr = P_<int32_t>(p, p.off.cost_ranges);
    const int32_t* wr = P_<int32_t>(p, p.off.cost_wave_ranges);
    const int32_t* wv = P_<int32_t>(p, p.off.cost_waves);
    const DevCostItem* items = P_<DevCostItem>(p, p.off.cost_items);
    const DevCostGate* CG = P_<DevCostGate>(p, p.off.cost_gates);
    const DevChannel* chans = P_<DevChannel>(p, p.off.channels);
    const double* cum = P_<double>(p, p.off.cum);
    bool count_near = true;
    if (p.hdr.has_frame && chain_clean<R>(p, ch)) {
        for (int it = cr[m] + G.lt; it < cr[m + 1]; it += G.nt)
            if (items[it].kind == CI_CHANNEL && kraus_pick<R>(p, ch, chans[items[it].idx], cum, sample_id, true) != 0)
                ch.misc[MISC_DIRTY_EVENT] = 1;
        G.sync();
        if (ch.misc[MISC_DIRTY_EVENT] == 0) return;
        // leaves the clean state in this section: segments m-1 .. P restart
        // from one (the earlier ones keep the fixed factors they hold)
        const int nseg = P1 - (m - 1);
        for (int i = G.lt; i < p.hdr.n * nseg * 2; i += G.nt) {
            const int q = i / (nseg * 2), r = i - q * nseg * 2;
            ch.segfac[((size_t)q * P1 + (m - 1)) * 2 + r] = mk<R>(1, 0);
        }
        if (G.lt == 0) ch.misc[MISC_CLEAN] = 0;
        count_near = false;   // these draws were counted above
        G.sync();
    }
    for (int w = wr[m]; w < wr[m + 1]; ++w) {
        for (int it = wv[w] + G.lt; it < wv[w + 1]; it += G.nt) {
            const DevCostItem ci = items[it];
            if (ci.kind == CI_GATE2) {
                ch.gframe[ci.idx] = (uint8_t)(ch.x[CG[ci.idx].q0] | (ch.x[CG[ci.idx].q1] << 1));
            } else if (ci.kind == CI_GATE1) {
                const int q = CG[ci.idx].q0, xb = ch.x[q];
                C* sf = ch.segfac + ((size_t)q * P1 + (m - 1)) * 2;
                sf[0] = cmul(sf[0], mk<R>((R)CG[ci.idx].d[2 * xb], (R)CG[ci.idx].d[2 * xb + 1]));
                sf[1] = cmul(sf[1], mk<R>((R)CG[ci.idx].d[2 * (1 ^ xb)], (R)CG[ci.idx].d[2 * (1 ^ xb) + 1]));
            } else if (p.mode == MODE_SAMPLE) {
                apply_channel<R>(p, ch, chans[ci.idx], cum, P_<DevKrausFactor>(p, p.off.factors), sample_id, m - 1,
                                 count_near);
            }
        }
        G.sync();
    }
}

// ---------------------------------------------------------------- chain
template <typename R>
__device__ void run_chain(const KParams& p, const Chain<R>& ch, int gid, int lt, uint64_t chain) {
    using C = typename CT<R>::T;
    const DevPlanHeader& h = p.hdr;
    const int n = h.n, P = h.P, S = h.S, K = h.K;
    const uint64_t sample_id = p.first + chain;
    const C one = mk<R>(1, 0);
    const DevBlockRange* BR = P_<DevBlockRange>(p, p.off.block_ranges);
    const Grp G{lt, p.tpc, gid, p.tpc, false, false};
    // amplitudes leave the kernel (trace, amplitude mode): keep every scale factor
    const bool exact = p.mode == MODE_AMP || p.trace != nullptr;

    for (int q = lt; q < n; q += p.tpc) {
        ch.x[q] = 0;
        ch.s[q] = p.mode == MODE_AMP ? (uint8_t)((p.in_bits[chain * h.words + (q >> 6)] >> (q & 63)) & 1ull) : 0;
    }
    if (h.has_frame) {
        for (int i = lt; i < (P + 1) * n; i += p.tpc) ch.xmix[i] = 0;
        for (int i = lt; i < h.n_cost_gates; i += p.tpc) ch.gframe[i] = 0;
    }
    if (h.has_segfac) {
        // a chain that starts clean holds the fixed segment factors of its
        // plan (one-qubit diagonal gates, Kraus operators 0); tables built at
        // run time read them from here
        const bool starts_clean = h.has_frame && h.clean_tables && p.mode == MODE_SAMPLE;
        const C* def = reinterpret_cast<const C*>(sizeof(R) == 4 ? P_<unsigned char>(p, p.off.segdef_f)
                                                                  : P_<unsigned char>(p, p.off.segdef_d));
        for (int i = lt; i < n * (P + 1) * 2; i += p.tpc) ch.segfac[i] = starts_clean ? def[i] : one;
    }
    if (lt == 0) {
        ch.misc[MISC_CLEAN] = 1;
        ch.misc[MISC_DIRTY_EVENT] = 0;
    }
    if (p.mode == MODE_SAMPLE) {
        // the UpdateState draws of every sampled gate (they depend only on
        // (seed, sample, op id), so they are drawn up front in parallel)
        const int32_t* rop = P_<int32_t>(p, p.off.row_opid);
        for (int r = lt; r < h.n_sampled; r += p.tpc) {
            const double u = draw_u(p.seed, sample_id, (uint32_t)rop[r], 0u);
            ch.ud[r] = u;
            ch.uf[r] = (float)u;
        }
        // Layer 0 acts on |0^n>: the prefix state is a product state, so the
        // conditional of qubit q is |<y|A_0|0>|^2 normalised (same draw rule).
        const int32_t* opid = P_<int32_t>(p, p.off.mix0_opid);
        const int8_t* mono = P_<int8_t>(p, p.off.mix_mono);
        const double* md = P_<double>(p, p.off.mix_d);
        for (int q = lt; q < n; q += p.tpc) {
            const double* A = md + (size_t)q * 8;
            if (mono[q]) {
                ch.s[q] = (A[0] != 0.0 || A[1] != 0.0) ? 0 : 1;
                continue;
            }
            const double p0 = A[0] * A[0] + A[1] * A[1];
            const double p1 = A[4] * A[4] + A[5] * A[5];
            const double Pt = p0 + p1;
            const double u = draw_u(p.seed, sample_id, (uint32_t)opid[q], 0u);
            ch.s[q] = (u * Pt < p0) ? 0 : 1;
            if (fabs(u * Pt - p0) < 1e-6 * Pt && ch.rank == 0) atomicAdd(&p.counters[CNT_NEAR], 1ull);
        }
    }
    G.sync();

    const int mhi = p.mode == MODE_AMP ? p.amp_layer : P;
    for (int m = 1; m <= mhi; ++m) {
        if (h.has_segfac || h.has_frame) {
            cost_section<R>(p, ch, G, m, sample_id);
            if (h.has_frame && !chain_clean<R>(p, ch))   // (a clean chain's frame rows stay zero)
                for (int q = lt; q < n; q += p.tpc) ch.xmix[m * n + q] = ch.x[q];
        }
        G.sync();
        if (p.mode == MODE_AMP && m < p.amp_layer) continue;

        const int Wl = S * (m - 1), W = S * m;
        const int NL = 1 << Wl, N = 1 << W;
        const int kstop = p.mode == MODE_AMP ? p.amp_block : 0;   // R_k needed for k >= kstop
        // small tensors run on the first warp only
        const int w32 = p.tpc < 32 ? p.tpc : 32;
        const bool dist = p.cr > 1 && W > p.wloc;   // frontier spread over the cluster
        // threads for a tensor of e entries: the whole group above 1024
        // entries (or when split over a cluster), four warps from 256 entries
        // when the group has at least 256 threads, else one warp
        auto phase_nt = [&](int e, bool d) { return (d || e > 1024) ? p.tpc : (e >= 256 && p.tpc >= 256) ? 128 : w32; };
        const int ntb = phase_nt(NL, false), ntf = phase_nt(N, dist);
        const Grp GB{lt, ntb, gid, p.tpc, ntb == 32 && p.tpc > 32, false};
        const Grp GF{lt, ntf, gid, p.tpc, ntf == 32 && p.tpc > 32, dist};

        // backward sweep: R_{K-1} = 1, R_{k-1} from R_k by block k's reversed
        // program. For m = 1 the environments are scalars (no summed segment on
        // the right), needed only for the exact scale.
        const bool skip_bwd = m == 1 && !exact;
        if (skip_bwd && lt < GB.nt) {
            for (int k = lt; k < K; k += GB.nt) {
                ch.Rt[k] = one;
                ch.Rexp[k] = 0;
            }
        }
        if (!skip_bwd && lt < GB.nt) {
            C* RK = ch.Rt + (size_t)(K - 1) * NL;
            for (int i = lt; i < NL; i += GB.nt) RK[i] = one;
            if (lt == 0) ch.Rexp[K - 1] = 0;
            for (int k = K - 1; k > kstop; --k) {
                const DevBlockRange br = BR[(size_t)m * K + k];
                const C* src = ch.Rt + (size_t)k * NL;
                C* dst = ch.Rt + (size_t)(k - 1) * NL;
                build_tables<R>(p, ch, GB, br.bwd_st, br.bwd_nst, br.bwd_tab, 0, exact);
                GB.sync();   // tables ready, previous environment complete
                for (int i = lt; i < NL; i += GB.nt) dst[i] = src[i];
                GB.sync();
                run_passes<R>(p, ch, GB, br.bwd_begin, br.bwd_end, br.bwd_st, dst, Wl);
                R mx = 0;
                for (int i = lt; i < NL; i += GB.nt) mx = rmax(mx, rmax(rabs(dst[i].x), rabs(dst[i].y)));
                mx = group_max<R>(ch, GB, mx);
                const int e = scale_exp<R>(mx);
                if (e != 0)
                    for (int i = lt; i < NL; i += GB.nt) {
                        dst[i].x = scl(dst[i].x, -e);
                        dst[i].y = scl(dst[i].y, -e);
                    }
                if (lt == 0) ch.Rexp[k - 1] = ch.Rexp[k] + e;
                GB.sync();
            }
        }
        G.sync();

        // forward sweep with a readout after every block
        if (lt < GF.nt) {
            const int Nl = dist ? (1 << p.wloc) : N;   // entries held by this CTA
            for (int i = lt; i < Nl; i += GF.nt) ch.L[i] = mk<R>(i == 0 && (!dist || ch.rank == 0) ? 1 : 0, 0);
            if (lt == 0) {
                ch.misc[0] = 0;
                ch.misc[1] = 0;
            }
            GF.sync();
            const int kend = p.mode == MODE_AMP ? p.amp_block : K - 1;
            for (int k = 0; k <= kend; ++k) {
                const DevBlockRange br = BR[(size_t)m * K + k];
                const int pend = ch.misc[1];
                build_tables<R>(p, ch, GF, br.fwd_st, br.fwd_nst, br.fwd_tab, pend, exact);
                build_fslot<R>(p, ch, GF, m, br);
                GF.sync();
                run_passes<R>(p, ch, GF, br.fwd_begin, br.fwd_end, br.fwd_st, ch.L, W, dist);
                readout_and_sample<R>(p, ch, GF, m, k, br, chain, dist);
            }
        }
        G.sync();
    }
    if (p.mode == MODE_AMP) return;

    // channels after the last layer (they can only move the frame)
    if (h.has_frame) cost_section<R>(p, ch, G, P + 1, sample_id);
    G.sync();
    // sample = s XOR x (Alg. 2), packed 64 qubits per word
    for (int w = lt; w < h.words && ch.rank == 0; w += p.tpc) {
        uint64_t v = 0;
        for (int b = 0; b < 64 && w * 64 + b < n; ++b) v |= (uint64_t)(ch.s[w * 64 + b] ^ ch.x[w * 64 + b]) << b;
        p.out_bits[chain * h.words + w] = v;
    }
    G.sync();
}

// The per-chain view of a group's shared memory.
template <typename R> __device__ __forceinline__ Chain<R> make_chain(const KParams& p, unsigned char* g) {
    using C = typename CT<R>::T;
    Chain<R> ch;
    ch.L = reinterpret_cast<C*>(g + p.sm.L);
    ch.Rt = reinterpret_cast<C*>(g + p.sm.R);
    ch.Rexp = reinterpret_cast<int*>(g + p.sm.Rexp);
    ch.rowdot = reinterpret_cast<C*>(g + p.sm.rowdot);
    ch.wt = reinterpret_cast<C*>(g + p.sm.wt);
    ch.T = reinterpret_cast<C*>(g + p.sm.T);
    ch.sa = reinterpret_cast<C*>(g + p.sm.sit);
    ch.sinfo = reinterpret_cast<int*>(ch.sa + 4 * p.hdr.max_block);
    ch.tab = reinterpret_cast<C*>(g + p.sm.tab);
    ch.stg = reinterpret_cast<DevStage*>(g + p.sm.stg);
    ch.ud = reinterpret_cast<double*>(g + p.sm.ud);
    ch.uf = reinterpret_cast<float*>(g + p.sm.uf);
    ch.part = reinterpret_cast<C*>(g + p.sm.part);
    ch.fslot = reinterpret_cast<C*>(g + p.sm.fslot);
    ch.red = reinterpret_cast<R*>(g + p.sm.red);
    ch.s = g + p.sm.s;
    ch.x = g + p.sm.x;
    ch.xmix = g + p.sm.xmix;
    ch.gframe = g + p.sm.gframe;
    ch.segfac = reinterpret_cast<C*>(g + p.sm.segfac);
    ch.misc = reinterpret_cast<int*>(g + p.sm.misc);
    ch.pd = reinterpret_cast<double2*>(g + p.sm.pd);
    ch.rL = reinterpret_cast<C**>(g + p.sm.rlp);
    ch.cmax = reinterpret_cast<float*>(g + p.sm.cmax);
    ch.rank = 0;
    return ch;
}

// ------------------------------------------------------------ HBM engine
// The dense operator of pass fi of block program br (HBM engine): the
// product of the pass's stages restricted to its tile bits, Op[t'][t] over
// the E = 2^KT tile settings, applied to the identity one column at a time.
// Column c is held by 256 / E threads of one warp, R = E^2 / 256 entries each
// (rows j R + i for thread part j): a 2x2 stage on a row bit below log2 R
// combines a thread's own entries, one on a higher bit exchanges entries with
// the partner thread (shuffles); a diagonal stage scales every entry. No
// shared memory and no barriers. Then the operator goes to HBM for the GEMM
// kernels, and the stages deferred to the epilogue (diagonal factors that
// read bits outside the tile) write their tables instead.
template <int LB, int R2>
__device__ __forceinline__ void mat_local(float2 (&x)[R2], float2 m00, float2 m01, float2 m10, float2 m11) {
#pragma unroll
    for (int i = 0; i < R2; ++i)
        if (!((i >> LB) & 1)) {
            const float2 x0 = x[i], x1 = x[i | (1 << LB)];
            x[i] = cfma(m00, x0, cmul(m01, x1));
            x[i | (1 << LB)] = cfma(m10, x0, cmul(m11, x1));
        }
}

template <int KT>
__device__ __forceinline__ void compose_pass(const KParams& p, const float2* tabs, const DevStage* stg,
                                             const DevBlockRange& br, int fi, uint64_t chain, int tid) {
    constexpr int E = 1 << KT, TPC = 256 / E, RR = E * E / 256;   // threads per column, entries per thread
    constexpr int LR = KT == 6 ? 4 : 2;                           // log2 RR: the thread's own row bits
    static_assert((1 << LR) == RR, "entries per thread");
    const DevFused f = P_<DevFused>(p, p.off.fused)[fi];
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    const int c = tid / TPC, j = tid % TPC;   // column, part (row bits LR..KT-1)
    float2 x[RR];
#pragma unroll
    for (int i = 0; i < RR; ++i) x[i] = (j * RR + i) == c ? one : zero;
    for (int s2 = 0; s2 < f.nst; ++s2) {
        const DevStage st = stg[f.st_begin - br.fwd_st + s2];
        const float2* tab = tabs + st.tab_off;
        if (st.type == ST_MAT) {
            const int a = st.arg;
            const float2 m00 = tab[0], m01 = tab[1], m10 = tab[2], m11 = tab[3];
            if (a < LR) {
                switch (a) {   // (a compile-time bit: the entries stay in registers)
                    case 0: mat_local<0, RR>(x, m00, m01, m10, m11); break;
                    case 1: mat_local<1, RR>(x, m00, m01, m10, m11); break;
                    case 2: if constexpr (LR > 2) mat_local<2, RR>(x, m00, m01, m10, m11); break;
                    case 3: if constexpr (LR > 3) mat_local<3, RR>(x, m00, m01, m10, m11); break;
                    default: break;
                }
            } else {
                const int bit = a - LR, hi = (j >> bit) & 1;
#pragma unroll
                for (int i = 0; i < RR; ++i) {
                    float2 y;
                    y.x = __shfl_xor_sync(0xffffffffu, x[i].x, 1 << bit);
                    y.y = __shfl_xor_sync(0xffffffffu, x[i].y, 1 << bit);
                    x[i] = hi ? cfma(m10, y, cmul(m11, x[i])) : cfma(m00, x[i], cmul(m01, y));
                }
            }
        } else if (!st.epi) {
            // the table index is linear over XOR in the row's bits: weight w[t]
            // of tile bit t (1 << q when it is the table's bit q), the
            // thread's part j contributing its bits' weights once (all indices
            // compile-time: no local-memory arrays)
            int w[KT];
#pragma unroll
            for (int t = 0; t < KT; ++t) {
                w[t] = 0;
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    if (q < st.arg && f.tbits[t] == st.dbits[q]) w[t] = 1 << q;
            }
            int ej = 0;
#pragma unroll
            for (int t = LR; t < KT; ++t) ej ^= ((j >> (t - LR)) & 1) ? w[t] : 0;
#pragma unroll
            for (int i = 0; i < RR; ++i) {
                int e = ej;
#pragma unroll
                for (int t = 0; t < LR; ++t) e ^= ((i >> t) & 1) ? w[t] : 0;
                x[i] = cmul(x[i], tab[e]);
            }
        }
    }
    const uint64_t slot = (uint64_t)(fi - br.fwd_begin) * p.nch + chain;
    float2* dst = static_cast<float2*>(p.gOps) + (slot << (2 * KT));
#pragma unroll
    for (int i = 0; i < RR; ++i) dst[(j * RR + i) * E + c] = x[i];
    // the epilogue's tables, in stage order, 32 entries each
    float2* gdiag = static_cast<float2*>(p.gDiag);
    int d = 0;
    for (int s2 = 0; s2 < f.nst; ++s2) {
        const DevStage st = stg[f.st_begin - br.fwd_st + s2];
        if (st.type != ST_DIAG || !st.epi) continue;
        const float2* tab = tabs + st.tab_off;
        if (tid < 32) gdiag[(slot * 4 + d) * 32 + tid] = tid < (1 << st.arg) ? tab[tid] : zero;
        ++d;
    }
}

// The chain program of the HBM engine: the same steps as run_chain, with the
// frontier and the right environments in HBM and the forward passes of the
// dense layers left to the GEMM kernels. A launch resumes every chain at
// yield point p.y_from (restoring its saved state), runs it to the next yield
// point (block k of a dense layer prepared: tables built, readout factors
// staged, the block's dense operators written) and saves its state; the host
// runs the block's passes and launches again. Yield points are numbered over
// the dense layers' blocks in order (p.ybase[m] = the first of layer m).
__device__ __forceinline__ void run_chain_hbm(const KParams& p, const Chain<float>& ch0, unsigned char* grp, int gid,
                                           int lt, uint64_t chain) {
    using R = float;
    using C = float2;
    const DevPlanHeader& h = p.hdr;
    const int n = h.n, P = h.P, S = h.S, K = h.K;
    const uint64_t sample_id = p.first + chain;
    const C one = mk<R>(1, 0);
    const DevBlockRange* BR = P_<DevBlockRange>(p, p.off.block_ranges);
    const Grp G{lt, p.tpc, gid, p.tpc, false, false};
    const bool exact = p.mode == MODE_AMP || p.trace != nullptr;
    Chain<R> ch = ch0;
    ch.Rt = static_cast<C*>(p.gR) + chain * p.strideR;
    uint4* saved = reinterpret_cast<uint4*>(p.gState + chain * (uint64_t)p.state_bytes);
    uint4* live = reinterpret_cast<uint4*>(grp + p.state_off);
    const int y0 = p.y_from;

    if (y0 >= 0) {
        for (int i = lt; i < p.state_bytes / 16; i += p.tpc) live[i] = saved[i];
        G.sync();
    } else {
        for (int q = lt; q < n; q += p.tpc) {
            ch.x[q] = 0;
            ch.s[q] = p.mode == MODE_AMP ? (uint8_t)((p.in_bits[chain * h.words + (q >> 6)] >> (q & 63)) & 1ull) : 0;
        }
        if (h.has_frame) {
            for (int i = lt; i < (P + 1) * n; i += p.tpc) ch.xmix[i] = 0;
            for (int i = lt; i < h.n_cost_gates; i += p.tpc) ch.gframe[i] = 0;
        }
        if (h.has_segfac) {
            const bool starts_clean = h.has_frame && h.clean_tables && p.mode == MODE_SAMPLE;
            const C* def = reinterpret_cast<const C*>(P_<unsigned char>(p, p.off.segdef_f));
            for (int i = lt; i < n * (P + 1) * 2; i += p.tpc) ch.segfac[i] = starts_clean ? def[i] : one;
        }
        if (lt == 0) {
            ch.misc[MISC_CLEAN] = 1;
            ch.misc[MISC_DIRTY_EVENT] = 0;
        }
        if (p.mode == MODE_SAMPLE) {
            const int32_t* rop = P_<int32_t>(p, p.off.row_opid);
            for (int r = lt; r < h.n_sampled; r += p.tpc) {
                const double u = draw_u(p.seed, sample_id, (uint32_t)rop[r], 0u);
                ch.ud[r] = u;
                ch.uf[r] = (float)u;
            }
            const int32_t* opid = P_<int32_t>(p, p.off.mix0_opid);
            const int8_t* mono = P_<int8_t>(p, p.off.mix_mono);
            const double* md = P_<double>(p, p.off.mix_d);
            for (int q = lt; q < n; q += p.tpc) {
                const double* A = md + (size_t)q * 8;
                if (mono[q]) {
                    ch.s[q] = (A[0] != 0.0 || A[1] != 0.0) ? 0 : 1;
                    continue;
                }
                const double p0 = A[0] * A[0] + A[1] * A[1];
                const double p1 = A[4] * A[4] + A[5] * A[5];
                const double Pt = p0 + p1;
                const double u = draw_u(p.seed, sample_id, (uint32_t)opid[q], 0u);
                ch.s[q] = (u * Pt < p0) ? 0 : 1;
                if (fabs(u * Pt - p0) < 1e-6 * Pt) atomicAdd(&p.counters[CNT_NEAR], 1ull);
            }
        }
        G.sync();
    }

    const int mhi = p.mode == MODE_AMP ? p.amp_layer : P;
    for (int m = 1; m <= mhi; ++m) {
        const bool skip_layer = p.mode == MODE_AMP && m < p.amp_layer;
        const bool dense = ((h.dense_mask >> m) & 1) && !skip_layer;
        const int kend = p.mode == MODE_AMP ? p.amp_block : K - 1;
        const int yb = p.ybase[m], ny = dense ? kend + 1 : 0;
        // layers behind the resume point ran in earlier launches
        if (y0 >= yb + ny && (ny > 0 || y0 >= yb)) continue;
        const bool resume_here = ny > 0 && y0 >= yb;
        const int Wl = S * (m - 1), W = S * m;
        const int NL = 1 << Wl, N = 1 << W;
        // a chain's frontier sits at the same place at every layer (stride of
        // the widest one): chains at different layers run concurrently
        ch.L = static_cast<C*>(p.gL) + chain * ((uint64_t)1 << (S * P));
        const int kstop = p.mode == MODE_AMP ? p.amp_block : 0;
        const int w32 = p.tpc < 32 ? p.tpc : 32;
        // (phases of 256 entries and more take the whole group: at four chains
        // per SM the group's other warps would otherwise idle)
        auto phase_nt = [&](int e) { return e >= 256 ? (p.tpc > 128 && e <= 1024 ? 128 : p.tpc) : w32; };
        const int ntb = phase_nt(NL), ntf = dense ? p.tpc : phase_nt(N);
        const Grp GB{lt, ntb, gid, p.tpc, ntb == 32 && p.tpc > 32, false};
        const Grp GF{lt, ntf, gid, p.tpc, ntf == 32 && p.tpc > 32, false};
        if (!resume_here) {
            if (h.has_segfac || h.has_frame) {
                cost_section<R>(p, ch, G, m, sample_id);
                if (h.has_frame && !chain_clean<R>(p, ch))
                    for (int q = lt; q < n; q += p.tpc) ch.xmix[m * n + q] = ch.x[q];
            }
            G.sync();
            if (skip_layer) continue;
            // backward sweep (right environments in HBM)
            const bool skip_bwd = m == 1 && !exact;
            if (skip_bwd && lt < GB.nt) {
                for (int k = lt; k < K; k += GB.nt) {
                    ch.Rt[k] = one;
                    ch.Rexp[k] = 0;
                }
            }
            if (!skip_bwd && lt < GB.nt) {
                C* RK = ch.Rt + (size_t)(K - 1) * NL;
                for (int i = lt; i < NL; i += GB.nt) RK[i] = one;
                if (lt == 0) ch.Rexp[K - 1] = 0;
                for (int k = K - 1; k > kstop; --k) {
                    const DevBlockRange br = BR[(size_t)m * K + k];
                    const C* src = ch.Rt + (size_t)k * NL;
                    C* dst = ch.Rt + (size_t)(k - 1) * NL;
                    build_tables<R>(p, ch, GB, br.bwd_st, br.bwd_nst, br.bwd_tab, 0, exact);
                    GB.sync();
                    for (int i = lt; i < NL; i += GB.nt) dst[i] = src[i];
                    GB.sync();
                    run_passes<R>(p, ch, GB, br.bwd_begin, br.bwd_end, br.bwd_st, dst, Wl);
                    R mx = 0;
                    for (int i = lt; i < NL; i += GB.nt) mx = rmax(mx, rmax(rabs(dst[i].x), rabs(dst[i].y)));
                    mx = group_max<R>(ch, GB, mx);
                    const int e = scale_exp<R>(mx);
                    if (e != 0)
                        for (int i = lt; i < NL; i += GB.nt) {
                            dst[i].x = scl(dst[i].x, -e);
                            dst[i].y = scl(dst[i].y, -e);
                        }
                    if (lt == 0) ch.Rexp[k - 1] = ch.Rexp[k] + e;
                    GB.sync();
                }
            }
            G.sync();
            if (lt < GF.nt) {
                for (int i = lt; i < N; i += GF.nt) ch.L[i] = mk<R>(i == 0 ? 1 : 0, 0);
                if (lt == 0) {
                    ch.misc[0] = 0;
                    ch.misc[1] = 0;
                }
            }
            G.sync();
        }
        if (lt < GF.nt) {
            const int kstart = resume_here ? y0 - yb : 0;
            for (int k = kstart; k <= kend; ++k) {
                const DevBlockRange br = BR[(size_t)m * K + k];
                if (!(resume_here && k == kstart)) {
                    const int pend = ch.misc[1];
                    build_tables<R>(p, ch, GF, br.fwd_st, br.fwd_nst, br.fwd_tab, pend, exact);
                    build_fslot<R>(p, ch, GF, m, br);
                    GF.sync();
                    if (dense) {
                        // yield: hbm_compose_kernel composes this block's operators
                        // from the saved tables, then the GEMM kernels run its passes
                        for (int i = lt; i < p.state_bytes / 16; i += p.tpc) saved[i] = live[i];
                        G.sync();
                        return;
                    }
                    run_passes<R>(p, ch, GF, br.fwd_begin, br.fwd_end, br.fwd_st, ch.L, W);
                }
                readout_and_sample<R>(p, ch, GF, m, k, br, chain);
            }
        }
        G.sync();
    }
    if (p.mode == MODE_AMP) return;
    if (h.has_frame) cost_section<R>(p, ch, G, P + 1, sample_id);
    G.sync();
    for (int w = lt; w < h.words; w += p.tpc) {
        uint64_t v = 0;
        for (int b = 0; b < 64 && w * 64 + b < n; ++b) v |= (uint64_t)(ch.s[w * 64 + b] ^ ch.x[w * 64 + b]) << b;
        p.out_bits[chain * h.words + w] = v;
    }
    G.sync();
}

// WIDE: the same kernel for CTAs of at most 64 threads with at most 5 of them
// per SM (the chains that shared memory admits on the 6x6 grid): up to 204
// registers per thread instead of 128, no occupancy lost when shared memory
// is the limit.
template <typename R, bool WIDE = false>
__global__ void __launch_bounds__(WIDE ? 64 : 512, WIDE ? 5 : 1) pw_chain_kernel(const KParams p) {
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    // The launches of one sampling call take disjoint chains and read only the
    // plan: the next one may start on the SMs this one no longer needs (it is
    // launched as a programmatic dependent of this one; elsewhere a no-op).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int gid = threadIdx.x / p.tpc;
    const int lt = threadIdx.x - gid * p.tpc;
    unsigned char* g = smem + (size_t)gid * p.sm.group_bytes;
    Chain<R> ch = make_chain<R>(p, g);
    if (p.cr > 1) {
        // one chain per cluster of p.cr CTAs (gpc == 1): every CTA keeps a copy
        // of the chain's small state and 1/cr of the frontier
        ch.rank = (int)__clusterRelativeBlockRank();
        if (lt < p.cr) ch.rL[lt] = static_cast<C*>(__cluster_map_shared_rank(ch.L, lt));
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        for (uint64_t chain = blockIdx.x / p.cr; chain < p.count; chain += gridDim.x / p.cr)
            run_chain<R>(p, ch, 0, lt, chain);
        // no CTA leaves while a peer may still read its shared memory
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        return;
    }
    ch.rank = 0;
    for (uint64_t chain = (uint64_t)blockIdx.x * p.gpc + gid; chain < p.count;
         chain += (uint64_t)gridDim.x * p.gpc)
        run_chain<R>(p, ch, gid, lt, chain);
}

// The HBM engine's chain kernel (FP32): one group of threads per chain, the
// chain program of run_chain_hbm from one yield point to the next.
__global__ void __launch_bounds__(512, 1) pw_chain_hbm_kernel(const KParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int gid = threadIdx.x / p.tpc;
    const int lt = threadIdx.x - gid * p.tpc;
    unsigned char* g = smem + (size_t)gid * p.sm.group_bytes;
    const Chain<float> ch = make_chain<float>(p, g);
    for (uint64_t chain = (uint64_t)blockIdx.x * p.gpc + gid; chain < p.count; chain += (uint64_t)gridDim.x * p.gpc)
        run_chain_hbm(p, ch, g, gid, lt, chain);
}

// The dense operators of one block of a dense layer for all chains of a
// batch (HBM engine). The block's stages (the same for every chain) are
// staged in shared memory once per CTA, a chain's tables (left by the chain
// kernel in its saved state) once per chain, all loads issued together; then
// each of the block's passes is composed in the registers of the CTA's 256
// threads.
__global__ void __launch_bounds__(256) hbm_compose_kernel(const KParams p, int m, int k, uint64_t cnt, int tab_at) {
    extern __shared__ __align__(16) unsigned char csm[];
    const DevBlockRange br = P_<DevBlockRange>(p, p.off.block_ranges)[(size_t)m * p.hdr.K + k];
    const DevFused* F = P_<DevFused>(p, p.off.fused);
    DevStage* sst = reinterpret_cast<DevStage*>(csm);
    float2* stab = reinterpret_cast<float2*>(csm + tab_at);
    const DevStage* gst = P_<DevStage>(p, p.off.stages) + br.fwd_st;
    for (int i = threadIdx.x; i < br.fwd_nst; i += 256) sst[i] = gst[i];
    for (uint64_t chain = blockIdx.x; chain < cnt; chain += gridDim.x) {
        const float2* tabs = reinterpret_cast<const float2*>(p.gState + chain * (uint64_t)p.state_bytes +
                                                             (p.sm.tab - p.state_off));
        __syncthreads();   // (the previous chain's tables are no longer read)
        for (int i = threadIdx.x; i < br.fwd_tab; i += 256) stab[i] = tabs[i];
        __syncthreads();
        for (int fi = br.fwd_begin; fi < br.fwd_end; ++fi) {
            if (F[fi].ntb == 6)
                compose_pass<6>(p, stab, sst, br, fi, chain, threadIdx.x);
            else
                compose_pass<5>(p, stab, sst, br, fi, chain, threadIdx.x);
        }
    }
}

// ================================================================= host
namespace {

template <typename T> void put(std::vector<unsigned char>& blob, int64_t& off, const std::vector<T>& v) {
    size_t at = align16(blob.size());
    blob.resize(at + std::max<size_t>(sizeof(T) * v.size(), 16));
    if (!v.empty()) std::memcpy(blob.data() + at, v.data(), sizeof(T) * v.size());
    off = (int64_t)at;
}

int cuda_fail(cudaError_t e, const char* what) {
    return set_error(PW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::vector<unsigned char> make_blob(const HostPlan& hp, DevPlanOffsets& o) {
    std::vector<unsigned char> blob;
    put(blob, o.micro, hp.micro);
    put(blob, o.fused, hp.fused);
    put(blob, o.stages, hp.stages);
    put(blob, o.row_opid, hp.row_opid);
    put(blob, o.vtab_f, hp.vtab_f);
    put(blob, o.vtab_d, hp.vtab_d);
    put(blob, o.gate_refs, hp.gate_refs);
    put(blob, o.cost_gates, hp.cost_gates);
    put(blob, o.cost_items, hp.cost_items);
    put(blob, o.cost_ranges, hp.cost_ranges);
    put(blob, o.cost_waves, hp.cost_waves);
    put(blob, o.cost_wave_ranges, hp.cost_wave_ranges);
    put(blob, o.channels, hp.channels);
    put(blob, o.cum, hp.cum);
    put(blob, o.factors, hp.factors);
    put(blob, o.mix_d, hp.mix_d);
    put(blob, o.mix_f, hp.mix_f);
    put(blob, o.mix0_order, hp.mix0_order);
    put(blob, o.mix0_opid, hp.mix0_opid);
    put(blob, o.mix_mono, hp.mix_mono);
    put(blob, o.segdef_d, hp.segdef_d);
    put(blob, o.segdef_f, hp.segdef_f);
    put(blob, o.block_ranges, hp.block_ranges);
    put(blob, o.block_sites, hp.block_sites);
    put(blob, o.live_slots, hp.live_slots);
    return blob;
}

int ensure_device_plan(pw_plan* plan) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (plan->d_blob && plan->device == dev) return PW_OK;
    if (plan->d_blob) {
        return set_error(PW_ERR_ARG, "plan was uploaded to another device; build one plan per device");
    }
    std::vector<unsigned char> blob = make_blob(plan->hp, plan->off);
    void* d = nullptr;
    if (int rc0 = dev_alloc(&d, blob.size(), "plan tables")) return rc0;
    // cudaMemcpy from pageable memory returns once the source is staged; the
    // copy itself is ordered on the legacy stream only. Wait for it, so that a
    // launch on any stream (also a non-blocking one) reads complete tables.
    if ((e = cudaMemcpy(d, blob.data(), blob.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess) {
        dev_free(d);
        return cuda_fail(e, "cudaMemcpy(plan)");
    }
    unsigned long long* cnt = nullptr;
    if (int rc0 = dev_alloc(reinterpret_cast<void**>(&cnt), 4 * sizeof(unsigned long long), "counters")) {
        dev_free(d);
        return rc0;
    }
    plan->d_blob = d;
    plan->blob_bytes = blob.size();
    plan->d_counters = cnt;
    plan->device = dev;
    return PW_OK;
}

// Shared-memory carveout for `resident` CTAs of `smem` bytes each: only what
// they need (plus the 1 KB the runtime reserves per CTA), so that the rest of
// the SM's unified L1 / shared storage stays L1, which caches the plan tables.
// The carveout is a preference that the driver rounds up to a supported size.
static int carveout_percent(int dev, int resident, size_t smem) {
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (maxsm <= 0 || resident <= 0) return 100;
    const size_t need = (size_t)resident * (smem + 1024);
    return (int)std::min<size_t>(100, (need * 100 + (size_t)maxsm - 1) / (size_t)maxsm);
}

// cudaFuncSetAttribute changes process-wide attributes of a kernel (its
// dynamic shared-memory limit, its carveout preference): every sequence of
// setting them, querying the occupancy they give and launching holds this
// lock, so that concurrent callers (the gradient lanes, other threads) cannot
// lower a limit between another caller's setting and its launch.
std::mutex& launch_mutex() {
    static std::mutex mu;
    return mu;
}

// Device buffers of the HBM engine for nch chains (kept by the plan and
// reused; enlarged when a call needs more chains).
struct HbmBuffers {
    size_t L, R, state, ops, diag, total;
};
HbmBuffers hbm_sizes(const HostPlan& hp, const SmemLayout& sm, uint64_t nch) {
    const int S = hp.hdr.S, P = std::max(hp.hdr.P, 1), K = std::max(hp.hdr.K, 1), k = std::max(hp.dense_k, 1);
    HbmBuffers b{};
    b.L = align16(nch * (sizeof(float2) << (S * P)));
    b.R = align16(nch * (size_t)K * (sizeof(float2) << (S * (P - 1))));
    b.state = align16(nch * (size_t)(sm.group_bytes - sm.R));
    b.ops = align16((size_t)std::max(hp.hdr.dense_npass, 1) * nch * (sizeof(float2) << (2 * k)));
    b.diag = align16((size_t)std::max(hp.hdr.dense_npass, 1) * nch * 4 * 32 * sizeof(float2));
    b.total = b.L + b.R + b.state + b.ops + b.diag;
    return b;
}

// The HBM engine: launches of the chain kernel that run every chain of a
// batch from one yield point to the next, with the dense passes of the
// prepared block (GEMMs on the frontiers in HBM) in between.
// Timing of the dense passes of one call (pw_sample with stats): an event
// pair around every pass, from the plan's pool.
struct DenseTiming {
    int used = 0;
    uint64_t passes = 0;
    double bytes = 0.0, flops = 0.0;
};

int launch_hbm(pw_plan* plan, KParams& kp, cudaStream_t st, uint64_t* launches, DenseTiming* tm) {
    const HostPlan& hp = plan->hp;
    const int S = hp.hdr.S, P = hp.hdr.P, K = hp.hdr.K;
    kp.sm = make_layout(hp, sizeof(float2));
    kp.tpc = hp.threads_per_chain;
    kp.cr = 1;
    kp.wloc = 0;
    kp.hbm = 1;
    if (kp.sm.group_bytes > 227 * 1024) return set_error(PW_ERR_TOO_LARGE, "per-chain shared memory exceeds 227 KB");
    const int gpc = groups_per_cta(kp.tpc, kp.sm.group_bytes);
    kp.gpc = gpc;
    const int threads = kp.tpc * gpc;
    const size_t smem = (size_t)kp.sm.group_bytes * gpc;
    void (*kern)(const KParams) = pw_chain_hbm_kernel;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int dev = plan->device, nsm = 0, occ = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    occ = std::max(occ, 1);
    // chains per batch: the plan's, else up to 8192 (and frontiers of at most 16 GB)
    const uint64_t by_mem = std::max<uint64_t>(1, (uint64_t(16) << 30) / (sizeof(float2) << (S * P)));
    const uint64_t per_launch = hp.chains_per_launch > 0 ? (uint64_t)hp.chains_per_launch
                                                         : std::min<uint64_t>({kp.count, 8192, by_mem});
    const HbmBuffers hb = hbm_sizes(hp, kp.sm, per_launch);
    if (!plan->d_dense || plan->dense_chains < per_launch) {
        if (plan->d_dense) dev_free(plan->d_dense);
        plan->d_dense = nullptr;
        plan->dense_chains = 0;
        if (int rc0 = dev_alloc(&plan->d_dense, hb.total, "HBM engine buffers")) return rc0;
        plan->dense_bytes = hb.total;
        plan->dense_chains = per_launch;
    }
    const uint64_t nch = plan->dense_chains;
    const HbmBuffers ha = hbm_sizes(hp, kp.sm, nch);
    unsigned char* base = static_cast<unsigned char*>(plan->d_dense);
    kp.gL = base;
    kp.gR = base + ha.L;
    kp.gState = base + ha.L + ha.R;
    kp.gOps = base + ha.L + ha.R + ha.state;
    kp.gDiag = base + ha.L + ha.R + ha.state + ha.ops;
    kp.strideR = (uint64_t)K << (S * std::max(P - 1, 0));
    kp.state_off = kp.sm.R;
    kp.state_bytes = kp.sm.group_bytes - kp.sm.R;
    kp.nch = nch;
    // yield points: every block of every dense layer that runs
    const int mhi = kp.mode == MODE_AMP ? kp.amp_layer : P;
    const int kend = kp.mode == MODE_AMP ? kp.amp_block : K - 1;
    std::vector<std::pair<int, int>> yields;
    for (int m = 1; m <= P && m < 8; ++m) {
        kp.ybase[m] = (int)yields.size();
        const bool dense = ((hp.hdr.dense_mask >> m) & 1) && m <= mhi && !(kp.mode == MODE_AMP && m < kp.amp_layer);
        if (dense)
            for (int k = 0; k <= kend; ++k) yields.push_back({m, k});
    }
    // the dense passes' arguments, per yield point
    const DevBlockRange* BRs = hp.block_ranges.data();
    const uint64_t total = kp.count, first0 = kp.first;
    uint64_t* out0 = kp.out_bits;
    double* tr0 = kp.trace;
    const uint64_t* in0 = kp.in_bits;
    double* amp0 = kp.amp_out;
    for (uint64_t done = 0; done < total; done += per_launch) {
        const uint64_t cnt = std::min(per_launch, total - done);
        kp.count = cnt;
        kp.first = first0 + done;
        kp.out_bits = out0 ? out0 + done * hp.hdr.words : nullptr;
        kp.trace = tr0 ? tr0 + done * (uint64_t)hp.hdr.n_sampled * 4 : nullptr;
        kp.in_bits = in0 ? in0 + done * hp.hdr.words : nullptr;
        kp.amp_out = amp0 ? amp0 + 2 * done : nullptr;
        const int grid = (int)std::min<uint64_t>((cnt + gpc - 1) / gpc, (uint64_t)nsm * occ);
        for (int y = -1; y < (int)yields.size(); ++y) {
            if (y >= 0) {
                const int m = yields[y].first, k = yields[y].second;
                const DevBlockRange& br = BRs[(size_t)m * K + k];
                {
                    // the block's operators, from the tables the chain kernel saved
                    const unsigned cgrid = (unsigned)std::min<uint64_t>(cnt, (uint64_t)nsm * 8);
                    const int tab_at = (int)align16(sizeof(DevStage) * (size_t)std::max(1, br.fwd_nst));
                    const size_t csm = (size_t)tab_at + sizeof(float2) * (size_t)std::max(1, br.fwd_tab);
                    if (csm > 227 * 1024) return set_error(PW_ERR_TOO_LARGE, "a block's tables exceed shared memory");
                    if (csm > 48 * 1024 &&
                        (e = cudaFuncSetAttribute(hbm_compose_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)csm)) != cudaSuccess)
                        return cuda_fail(e, "cudaFuncSetAttribute(compose)");
                    hbm_compose_kernel<<<cgrid, 256, csm, st>>>(kp, m, k, cnt, tab_at);
                    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "compose launch");
                    if (launches) ++*launches;
                }
                for (int fi = br.fwd_begin; fi < br.fwd_end; ++fi) {
                    const DevFused& f = hp.fused[fi];
                    const int pi = fi - br.fwd_begin;
                    DenseArgs a;
                    std::memset(&a, 0, sizeof(a));
                    a.L = static_cast<float2*>(kp.gL);
                    a.ntens = cnt;
                    a.W = S * m;
                    a.stride = (uint64_t)1 << (S * P);   // a chain's frontier keeps its place at every layer
                    a.k = f.ntb;
                    a.swz = 1;
                    for (int j = 0; j < a.k; ++j) a.tile_pos[j] = f.tbits[j];
                    // rows: the lowest live legs; tiles: the other live legs (a tile
                    // with a dead leg set holds zeros and is skipped)
                    a.nouter = dense_pass_bits(hp, fi, a.W, a.row_pos, a.outer_pos);
                    for (int s2 = 0; s2 < f.nst; ++s2) {
                        const DevStage& sg = hp.stages[f.st_begin + s2];
                        if (sg.type != ST_DIAG || !sg.epi) continue;
                        a.diag_nb[a.ndiag] = sg.arg;
                        for (int j = 0; j < sg.arg; ++j) a.diag_pos[a.ndiag][j] = sg.dbits[j];
                        ++a.ndiag;
                    }
                    a.ops = static_cast<const float2*>(kp.gOps) + (((uint64_t)pi * nch) << (2 * a.k));
                    a.diag = static_cast<const float2*>(kp.gDiag) + (uint64_t)pi * nch * 4 * 32;
                    a.diag_stride = 4 * 32;
                    a.err = reinterpret_cast<int*>(kp.counters + CNT_DENSE);
                    cudaEvent_t e0 = nullptr, e1 = nullptr;
                    if (tm) {
                        while ((int)plan->dense_events.size() < 2 * (tm->used + 1)) {
                            cudaEvent_t ev;
                            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
                            plan->dense_events.push_back(ev);
                        }
                        e0 = static_cast<cudaEvent_t>(plan->dense_events[2 * tm->used]);
                        e1 = static_cast<cudaEvent_t>(plan->dense_events[2 * tm->used + 1]);
                        ++tm->used;
                    }
                    // (the events bracket the GEMM kernel alone)
                    const int rc = dense_run(hp.gemm, a, st, e0, e1);
                    if (rc) return rc;
                    if (tm) {
                        const double entries = (double)cnt * std::ldexp(1.0, a.k + 7 + a.nouter);
                        const int nprod = hp.gemm == PW_GEMM_SPLIT3 ? 6 : hp.gemm == PW_GEMM_SPLIT2 ? 3 : 1;
                        ++tm->passes;
                        tm->bytes += 16.0 * entries;
                        tm->flops += 8.0 * entries * std::ldexp(1.0, a.k) * nprod;
                    }
                    if (launches) ++*launches;
                }
            }
            kp.y_from = y;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)grid);
            cfg.blockDim = dim3((unsigned)threads);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = st;
            e = cudaLaunchKernelEx(&cfg, kern, kp);
            if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
            if (launches) ++*launches;
        }
    }
    return PW_OK;
}

template <typename R> int launch(pw_plan* plan, KParams& kp, cudaStream_t st, uint64_t* launches,
                                 DenseTiming* tm = nullptr) {
    std::lock_guard<std::mutex> attr_lock(launch_mutex());
    if constexpr (sizeof(R) == 4) {
        if (plan->hp.engine == 1) return launch_hbm(plan, kp, st, launches, tm);
    }
    const HostPlan& hp = plan->hp;
    const size_t csz = 2 * sizeof(R);
    kp.sm = make_layout(hp, csz);
    kp.tpc = hp.threads_per_chain;
    // groups per CTA: as many as fit 227 KB of shared memory, at most 8
    const int maxsm = 227 * 1024;
    if (kp.sm.group_bytes > maxsm)
        return set_error(PW_ERR_TOO_LARGE, "per-chain shared memory (" + std::to_string(kp.sm.group_bytes) +
                                               " B) exceeds 227 KB");
    void (*kern)(const KParams) = pw_chain_kernel<R, false>;
    cudaError_t e;
    if (hp.ctas_per_chain > 1) {
        // one chain per thread-block cluster
        kp.cr = hp.ctas_per_chain;
        kp.wloc = hp.wloc;
        kp.gpc = 1;
        const size_t smem = (size_t)kp.sm.group_bytes;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)kp.cr;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.blockDim = dim3((unsigned)kp.tpc);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3((unsigned)kp.cr);
        int maxc = 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        e = cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveClusters");
        if (maxc < 1) return set_error(PW_ERR_TOO_LARGE, "no cluster of this size fits on the device");
        {
            // one CTA per SM: the carveout it needs, if that keeps every cluster
            int maxc2 = 0;
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 carveout_percent(plan->device, 1, smem));
            if (cudaOccupancyMaxActiveClusters(&maxc2, kern, &cfg) != cudaSuccess || maxc2 < maxc)
                cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        }
        const uint64_t per_launch = hp.chains_per_launch > 0 ? (uint64_t)hp.chains_per_launch : kp.count;
        const uint64_t total = kp.count, first0 = kp.first;
        uint64_t* out0 = kp.out_bits;
        double* tr0 = kp.trace;
        const uint64_t* in0 = kp.in_bits;
        double* amp0 = kp.amp_out;
        for (uint64_t done = 0; done < total; done += per_launch) {
            const uint64_t cnt = std::min(per_launch, total - done);
            kp.count = cnt;
            kp.first = first0 + done;
            kp.out_bits = out0 ? out0 + done * hp.hdr.words : nullptr;
            kp.trace = tr0 ? tr0 + done * (uint64_t)hp.hdr.n_sampled * 4 : nullptr;
            kp.in_bits = in0 ? in0 + done * hp.hdr.words : nullptr;
            kp.amp_out = amp0 ? amp0 + 2 * done : nullptr;
            cfg.gridDim = dim3((unsigned)(std::min<uint64_t>(cnt, (uint64_t)maxc) * kp.cr));
            cfg.numAttrs = done > 0 ? 2 : 1;   // later launches: programmatic dependents (see the kernel)
            e = cudaLaunchKernelEx(&cfg, kern, kp);
            if (e != cudaSuccess) return cuda_fail(e, "cluster kernel launch");
            if (launches) ++*launches;
        }
        return PW_OK;
    }
    kp.cr = 1;
    kp.wloc = 0;
    const int gpc = groups_per_cta(kp.tpc, kp.sm.group_bytes);
    kp.gpc = gpc;
    const int threads = kp.tpc * gpc;
    const size_t smem = (size_t)kp.sm.group_bytes * gpc;
    if constexpr (sizeof(R) == 4) {
        // the wide-register build when it keeps at least as many CTAs per SM
        if (threads <= 64) {
            auto wide = pw_chain_kernel<R, true>;
            int on = 0, ow = 0;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
                cudaFuncSetAttribute(wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
                cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess &&
                cudaFuncSetAttribute(wide, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&on, kern, threads, smem) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ow, wide, threads, smem) == cudaSuccess && ow >= on)
                kern = wide;
            cudaGetLastError();
        }
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int dev = plan->device, nsm = 0, occ = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    occ = std::max(occ, 1);
    {
        int occ2 = 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carveout_percent(dev, occ, smem));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, kern, threads, smem) != cudaSuccess || occ2 < occ)
            cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    const uint64_t per_launch = hp.chains_per_launch > 0 ? (uint64_t)hp.chains_per_launch : kp.count;
    const uint64_t total = kp.count, first0 = kp.first;
    uint64_t* out0 = kp.out_bits;
    double* tr0 = kp.trace;
    const uint64_t* in0 = kp.in_bits;
    double* amp0 = kp.amp_out;
    for (uint64_t done = 0; done < total; done += per_launch) {
        const uint64_t cnt = std::min(per_launch, total - done);
        kp.count = cnt;
        kp.first = first0 + done;
        kp.out_bits = out0 ? out0 + done * hp.hdr.words : nullptr;
        kp.trace = tr0 ? tr0 + done * (uint64_t)hp.hdr.n_sampled * 4 : nullptr;
        kp.in_bits = in0 ? in0 + done * hp.hdr.words : nullptr;
        kp.amp_out = amp0 ? amp0 + 2 * done : nullptr;
        const uint64_t ctas_needed = (cnt + gpc - 1) / gpc;
        const int grid = (int)std::min<uint64_t>(ctas_needed, (uint64_t)nsm * occ);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute pdl[1];
        pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        pdl[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl;
        cfg.numAttrs = done > 0 ? 1 : 0;   // the first launch waits for all earlier work
        e = cudaLaunchKernelEx(&cfg, kern, kp);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        if (launches) ++*launches;
    }
    return PW_OK;
}

int run(pw_plan* plan, KParams& kp, cudaStream_t st, uint64_t* launches, DenseTiming* tm = nullptr) {
    return plan->hp.precision == PW_PREC_FP64 ? launch<double>(plan, kp, st, launches)
                                              : launch<float>(plan, kp, st, launches, tm);
}

void fill_common(pw_plan* plan, KParams& kp) {
    std::memset(&kp, 0, sizeof(kp));
    kp.blob = static_cast<const unsigned char*>(plan->d_blob);
    kp.off = plan->off;
    kp.hdr = plan->hp.hdr;
    kp.counters = plan->d_counters;
}

}  // namespace

size_t plan_device_bytes(const HostPlan& hp) {
    DevPlanOffsets o;
    return make_blob(hp, o).size();
}
}  // namespace pw

using namespace pw;

extern "C" {

int pw_sample(pw_plan* plan, uint64_t seed, uint64_t first_sample, uint64_t n_samples, uint64_t* d_out_bits,
              double* d_trace, void* stream, pw_run_stats_t* stats) {
    if (!plan || (!d_out_bits && n_samples)) return set_error(PW_ERR_ARG, "null argument");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n_samples == 0) return PW_OK;
    int rc = ensure_device_plan(plan);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(plan->d_counters, 0, 4 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    KParams kp;
    fill_common(plan, kp);
    kp.seed = seed;
    kp.first = first_sample;
    kp.count = n_samples;
    kp.out_bits = d_out_bits;
    kp.trace = d_trace;
    kp.mode = MODE_SAMPLE;
    uint64_t launches = 0;
    DenseTiming tm;
    rc = run(plan, kp, st, &launches, stats ? &tm : nullptr);
    if (rc) return rc;
    if (!plan->out_wire.empty()) {   // wires back to qubits (SWAP-class gates)
        if ((rc = permute_output(plan, d_out_bits, n_samples, st))) return rc;
        ++launches;
    }
    if (stats) {
        unsigned long long h[4] = {0, 0, 0, 0};
        e = cudaMemcpyAsync(h, plan->d_counters, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading counters");
        stats->near_boundary = h[CNT_NEAR];
        stats->zero_mass = h[CNT_ZERO];
        stats->launches = launches;
        stats->dense_passes = tm.passes;
        stats->dense_bytes = tm.bytes;
        stats->dense_flops = tm.flops;
        double ms = 0.0;
        for (int i = 0; i < tm.used; ++i) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, static_cast<cudaEvent_t>(plan->dense_events[2 * i]),
                                     static_cast<cudaEvent_t>(plan->dense_events[2 * i + 1])) == cudaSuccess)
                ms += t;
        }
        stats->dense_ms = ms;
        if (h[CNT_DENSE]) return set_error(PW_ERR_TIMEOUT, "a bounded wait of a tensor-core pass ran out");
    }
    return PW_OK;
}

int pw_plan_autotune(pw_plan* plan, uint64_t trial_samples, void* stream, int* chosen) {
    if (!plan) return set_error(PW_ERR_ARG, "null argument");
    HostPlan& hp = plan->hp;
    const int keep = hp.threads_per_chain;
    if (chosen) *chosen = keep;
    if (hp.ctas_per_chain > 1 || hp.engine == 1) return PW_OK;   // clusters and the HBM engine keep their shape
    int rc = ensure_device_plan(plan);
    if (rc) return rc;
    const uint64_t cpl = hp.chains_per_launch > 0 ? (uint64_t)hp.chains_per_launch : 4096;
    const uint64_t n = trial_samples ? trial_samples : 4 * cpl;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t* d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (int rc0 = dev_alloc(reinterpret_cast<void**>(&d_out), n * hp.hdr.words * sizeof(uint64_t), "autotune output")) return rc0;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        if (d_out) dev_free(d_out);
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(e, "autotune set-up");
    }
    int best = keep;
    float best_ms = 0.0f;
    for (int tpc = 32; tpc <= 256; tpc *= 2) {
        hp.threads_per_chain = tpc;
        // one warm-up call, then the fastest of three timed ones
        rc = pw_sample(plan, 0x5eed, 0, n, d_out, nullptr, stream, nullptr);
        float ms = 0.0f;
        for (int rep = 0; rep < 3 && rc == PW_OK; ++rep) {
            cudaEventRecord(e0, st);
            rc = pw_sample(plan, 0x5eed, (rep + 1) * n, n, d_out, nullptr, stream, nullptr);
            cudaEventRecord(e1, st);
            float t = 0.0f;
            if (rc == PW_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
                ms = (rep == 0 || t < ms) ? t : ms;
            else
                rc = PW_ERR_CUDA;
        }
        if (rc == PW_OK && ms > 0.0f && (best_ms == 0.0f || ms < best_ms)) {
            best_ms = ms;
            best = tpc;
        }
        cudaGetLastError();   // (a configuration that does not fit is skipped)
    }
    hp.threads_per_chain = best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(d_out);
    if (best_ms == 0.0f) {
        hp.threads_per_chain = keep;
        return set_error(PW_ERR_CUDA, "autotune: no configuration ran");
    }
    if (chosen) *chosen = best;
    return PW_OK;
}

int pw_sample_host(pw_plan* plan, uint64_t seed, uint64_t first_sample, uint64_t n_samples, uint64_t* h_out_bits,
                   double* h_trace, pw_run_stats_t* stats) {
    if (!plan || (!h_out_bits && n_samples)) return set_error(PW_ERR_ARG, "null argument");
    if (n_samples == 0) {
        if (stats) std::memset(stats, 0, sizeof(*stats));
        return PW_OK;
    }
    int rc = ensure_device_plan(plan);
    if (rc) return rc;
    const size_t bits_bytes = (size_t)n_samples * plan->hp.hdr.words * sizeof(uint64_t);
    const size_t tr_bytes = h_trace ? (size_t)n_samples * plan->hp.hdr.n_sampled * 4 * sizeof(double) : 0;
    const size_t need = align16(bits_bytes) + tr_bytes;
    cudaError_t e;
    if (plan->stage_bytes < need) {
        if (plan->d_stage) dev_free(plan->d_stage);
        plan->d_stage = nullptr;
        plan->stage_bytes = 0;
        if (int rc0 = dev_alloc(&plan->d_stage, need, "staging")) return rc0;
        plan->stage_bytes = need;
    }
    uint64_t* d_bits = static_cast<uint64_t*>(plan->d_stage);
    double* d_tr = h_trace ? reinterpret_cast<double*>(static_cast<unsigned char*>(plan->d_stage) + align16(bits_bytes))
                           : nullptr;
    pw_run_stats_t local;
    rc = pw_sample(plan, seed, first_sample, n_samples, d_bits, d_tr, nullptr, &local);
    if (rc) return rc;
    if ((e = cudaMemcpy(h_out_bits, d_bits, bits_bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy(bits)");
    if (h_trace && (e = cudaMemcpy(h_trace, d_tr, tr_bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy(trace)");
    if (stats) *stats = local;
    return PW_OK;
}

int pw_amplitudes(pw_plan* plan, int prefix_ops, uint64_t n_strings, const uint64_t* d_bits, double* d_amp,
                  void* stream) {
    if (!plan || ((!d_bits || !d_amp) && n_strings)) return set_error(PW_ERR_ARG, "null argument");
    const HostPlan& hp = plan->hp;
    if (hp.noisy) return set_error(PW_ERR_UNSUPPORTED, "amplitudes are defined for noiseless circuits only");
    const bool relabelled = !plan->out_wire.empty();
    if (relabelled && prefix_ops != (int)hp.exec_order.size())
        return set_error(PW_ERR_UNSUPPORTED,
                         "with SWAP-class gates only the amplitudes of the whole circuit are supported");
    if (prefix_ops < 1 || prefix_ops > (int)hp.exec_order.size()) return set_error(PW_ERR_ARG, "prefix_ops out of range");
    const int op = hp.exec_order[prefix_ops - 1];
    if (hp.exec_layer[op] < 1)
        return set_error(PW_ERR_ARG, "the prefix must end right after a one-qubit gate of a layer >= 1");
    if (n_strings == 0) return PW_OK;
    int rc = ensure_device_plan(plan);
    if (rc) return rc;
    KParams kp;
    fill_common(plan, kp);
    kp.count = n_strings;
    kp.mode = MODE_AMP;
    kp.in_bits = d_bits;
    kp.amp_out = d_amp;
    kp.amp_layer = hp.exec_layer[op];
    kp.amp_block = hp.exec_block[op];
    kp.amp_pos = hp.exec_pos[op];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(plan->d_counters, 0, 4 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (!relabelled) return run(plan, kp, st, nullptr);
    // the kernel reads the bits per wire: reorder a copy of the strings
    uint64_t* d_wire_bits = nullptr;
    if ((rc = dev_alloc(reinterpret_cast<void**>(&d_wire_bits), n_strings * hp.hdr.words * sizeof(uint64_t),
                        "wire-ordered strings")))
        return rc;
    rc = permute_input(plan, d_bits, d_wire_bits, n_strings, st);
    if (!rc) {
        kp.in_bits = d_wire_bits;
        rc = run(plan, kp, st, nullptr);
    }
    e = cudaStreamSynchronize(st);   // before the copy is freed
    dev_free(d_wire_bits);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
    return rc;
}

}  // extern "C"

// =============================================== allocation-free sampling
// pw_sample_static: the same sampler for callers that cannot allocate device
// memory (for example a process whose device memory is entirely reserved by a
// framework's own pool, or a loop that must not allocate). The kernel's scratch
// (the plan tables it reads and its two draw counters) lives in one file-scope
// device array of fixed size instead of library allocations.
namespace pw {
namespace {

constexpr size_t kStaticScratchBytes = size_t(2) << 20;   // 2 MiB per device
constexpr size_t kStaticCounterBytes = 256;               // counters, then plan tables

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, looked up once per device
// with that device current (the host symbol is only a stand-in).
std::mutex g_static_mu;
void* g_static_ptr[64] = {nullptr};

int static_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= 64) return set_error(PW_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[dev] = ptr;
    }
    *out = static_cast<unsigned char*>(g_static_ptr[dev]);
    return PW_OK;
}

template <typename R> int launch_static(const HostPlan& hp, int dev, KParams& kp, cudaStream_t st, uint64_t* launches) {
    std::lock_guard<std::mutex> attr_lock(launch_mutex());
    kp.sm = make_layout(hp, 2 * sizeof(R));
    kp.tpc = hp.threads_per_chain;
    if (kp.sm.group_bytes > 227 * 1024) return set_error(PW_ERR_TOO_LARGE, "per-chain shared memory exceeds 227 KB");
    const int gpc = groups_per_cta(kp.tpc, kp.sm.group_bytes);
    kp.gpc = gpc;
    const int threads = kp.tpc * gpc;
    const size_t smem = (size_t)kp.sm.group_bytes * gpc;
    auto kern = pw_chain_kernel<R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int nsm = 0, occ = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    occ = std::max(occ, 1);
    const uint64_t per_launch = hp.chains_per_launch > 0 ? (uint64_t)hp.chains_per_launch : kp.count;
    const uint64_t total = kp.count, first0 = kp.first;
    uint64_t* out0 = kp.out_bits;
    for (uint64_t done = 0; done < total; done += per_launch) {
        const uint64_t cnt = std::min(per_launch, total - done);
        kp.count = cnt;
        kp.first = first0 + done;
        kp.out_bits = out0 + done * hp.hdr.words;
        const int grid = (int)std::min<uint64_t>((cnt + gpc - 1) / gpc, (uint64_t)nsm * occ);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute pdl[1];
        pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        pdl[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl;
        cfg.numAttrs = done > 0 ? 1 : 0;   // the first launch waits for all earlier work
        e = cudaLaunchKernelEx(&cfg, kern, kp);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        if (launches) ++*launches;
    }
    return PW_OK;
}

}  // namespace
}  // namespace pw

extern "C" int pw_sample_static(const pw_plan* plan, uint64_t seed, uint64_t first_sample, uint64_t n_samples,
                                uint64_t* d_out_bits, void* stream, pw_run_stats_t* stats) {
    using namespace pw;
    if (!plan || (!d_out_bits && n_samples)) return set_error(PW_ERR_ARG, "null argument");
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n_samples == 0) return PW_OK;
    const HostPlan& hp = plan->hp;
    if (hp.ctas_per_chain > 1 || hp.engine == 1)
        return set_error(PW_ERR_UNSUPPORTED, "pw_sample_static runs on-chip plans of one CTA per chain only");
    if (!plan->out_wire.empty())
        return set_error(PW_ERR_UNSUPPORTED, "pw_sample_static does not run circuits with SWAP-class gates");
    DevPlanOffsets off{};
    const std::vector<unsigned char> blob = make_blob(hp, off);
    if (blob.size() > kStaticScratchBytes - kStaticCounterBytes)
        return set_error(PW_ERR_TOO_LARGE, "plan tables (" + std::to_string(blob.size()) +
                                               " B) exceed the static scratch of pw_sample_static (" +
                                               std::to_string(kStaticScratchBytes - kStaticCounterBytes) + " B)");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char* base = nullptr;
    int rc = static_scratch(dev, &base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: reload the tables, zero the counters
    e = cudaMemcpyAsync(base + kStaticCounterBytes, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, kStaticCounterBytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "staging the plan tables");
    KParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.blob = base + kStaticCounterBytes;
    kp.off = off;
    kp.hdr = hp.hdr;
    kp.counters = reinterpret_cast<unsigned long long*>(base);
    kp.seed = seed;
    kp.first = first_sample;
    kp.count = n_samples;
    kp.out_bits = d_out_bits;
    kp.mode = MODE_SAMPLE;
    kp.cr = 1;
    uint64_t launches = 0;
    rc = hp.precision == PW_PREC_FP64 ? launch_static<double>(hp, dev, kp, st, &launches)
                                      : launch_static<float>(hp, dev, kp, st, &launches);
    if (rc) return rc;
    if (stats) {
        unsigned long long hcnt[4] = {0, 0, 0, 0};
        e = cudaMemcpyAsync(hcnt, base, sizeof(hcnt), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading counters");
        stats->near_boundary = hcnt[CNT_NEAR];
        stats->zero_mass = hcnt[CNT_ZERO];
        stats->launches = launches;
    }
    return PW_OK;
}

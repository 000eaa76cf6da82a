// Dense passes of the sweep contraction on an HBM-resident frontier.
//
// A pass of the plan's sweep (Sec. 2: the amplitudes amp(C_t, y) are
// contractions of the circuit's tensor network) applies a product of 2x2
// matrices on a few index bits of a chain's frontier tensor and of diagonal
// factors. Composed over k tile bits it is one dense 2^k x 2^k complex
// operator Op (per chain) followed by diagonal factors that also read other
// bits. With the tensor of 2^W entries in HBM, the pass is a GEMM:
//   rows    = the 2^(W-k) settings of the other bits (M, in tiles of 128),
//   columns = the 2^k settings of the tile bits (K in, N out),
// y[row, t'] = D(row, t') * sum_t x[row, t] Op[t'][t], complex, in place.
// Complex numbers enter the real GEMM as 2x2 real blocks: row entries
// interleave (re, im) and the operator becomes Bre[2t'+c'][2t+c] =
// [[Re, -Im], [Im, Re]] of Op[t'][t], so K = N = 2^(k+1) reals.
//
// Two arms run the same pass:
//   * dense_tc_kernel: 5th-generation tensor cores (tcgen05.mma, kind::f16,
//     BF16 operands, FP32 accumulators in tensor memory). FP32 operands are
//     split into NP BF16 terms x = x_0 + x_1 (+ x_2) (8 significant bits
//     each) and the products of total order below NP are accumulated: one
//     product for NP = 1 (plain BF16), three for NP = 2, six for NP = 3
//     (inputs represented to 24 bits, the FP32 significand). One warp issues
//     the MMAs, eight producer warps gather the A tiles (rows of 2^k entries
//     at scattered index bits) and write the BF16 terms into shared memory in
//     the 128-byte-swizzled K-major layout, eight epilogue warps (two per
//     quarter of the accumulator lanes) read the accumulators back
//     (tcgen05.ld) and scatter the rows to HBM. The B
//     operand (one per tensor) is split into its BF16 term planes by the
//     producers, from the operator's FP32 copy in HBM, whenever the tile
//     sequence of a CTA reaches the next tensor.
//   * dense_simt_kernel: the same GEMM on FP32 CUDA cores (the plain-FP32
//     comparison arm).
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "dense.h"
#include "pw_internal.h"

namespace pw {
namespace {

constexpr long long kWaitCycles = 4000000000ll;   // bounded waits: about 2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete; false (and the CTA's
// abort flag set) when it did not within kWaitCycles, or when another role
// of the CTA gave up already.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > kWaitCycles) {
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: 128-byte swizzle, K-major, 8-row groups
// 1024 bytes apart (stride byte offset), fixed field 0b001 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;      // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;               // SWIZZLE_128B
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 lanes x 256 bits of 32-bit accumulators, repeated along the columns
// (NREP = 4 or 8: 32 or 64 columns): thread t holds lane t / 4 in registers
// 4 i and 4 i + 1, lane t / 4 + 8 in 4 i + 2 and 4 i + 3, at columns
// col + 8 i + 2 (t % 4) and + 1 (the accumulator fragment of a 16-row MMA).
template <int NREP> __device__ __forceinline__ void tmem_ld16x256(uint32_t taddr, float (&v)[4 * NREP]) {
    uint32_t r[4 * NREP];
    if constexpr (NREP == 8) {
        asm volatile(
            "tcgen05.ld.sync.aligned.16x256b.x8.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr)
            : "memory");
    } else {
        static_assert(NREP == 4, "16x256b loads of 4 or 8 repetitions");
        asm volatile(
            "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 4 * NREP; ++j) v[j] = __uint_as_float(r[j]);
}

// The BF16 terms of a pair (x, y), converted together (round to nearest at
// every step): x = t0 + t1 (+ t2) exactly for NP = 3 (the 24 significant bits
// of an FP32 value), to about 2^-17 |x| for NP = 2. Word q holds term q of x
// in its low half and of y in its high half.
template <int NP> __device__ __forceinline__ void split_pair(float x, float y, uint32_t (&w)[NP]) {
    float2 r = make_float2(x, y);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        const __nv_bfloat162 t = __float22bfloat162_rn(r);
        w[q] = *reinterpret_cast<const uint32_t*>(&t);
        if (q + 1 < NP) {
            const float2 f = __bfloat1622float2(t);
            r.x -= f.x;
            r.y -= f.y;
        }
    }
}

// Word j of every term plane: the BF16 terms of (re, im) side by side (re in
// the low half: k index 2j before 2j + 1).
template <int NP> __device__ __forceinline__ void pack_terms(float re, float im, uint32_t (&h)[NP][4], int j) {
    uint32_t w[NP];
    split_pair<NP>(re, im, w);
#pragma unroll
    for (int q = 0; q < NP; ++q) h[q][j] = w[q];
}

// Byte offset of the 16-byte chunk c (8 BF16 values, k index 8c..8c+7 of the
// 64 in one 128-byte row segment) of row r in a K-major, 128-byte-swizzled
// operand of `rows` rows: K blocks of 64 values are rows x 128 bytes apart.
__device__ __forceinline__ uint32_t sw128_chunk(int rows, int r, int kb, int c) {
    return (uint32_t)(kb * rows * 128 + r * 128 + ((c ^ (r & 7)) << 4));
}

// Byte offset of complex entry (row r, column c) of the A operand: the
// 4-byte (re, im) pair of c in its 16-byte chunk (c >> 2) & 7. Every field is
// an XOR of bits of r and c (bits 2, 3: c; 4..6: c ^ r; 7..13: r; 14: c), so
// the offsets of disjoint bit sets combine by XOR.
__device__ __forceinline__ int a_offset(int r, int c) {
    return (int)sw128_chunk(128, r, c >> 5, (c >> 2) & 7) + ((c & 3) << 2);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ int64_t outer_offset(const DenseArgs& a, uint64_t o) {
    int64_t off = 0;
    for (int b = 0; b < a.nouter; ++b) off |= (int64_t)((o >> b) & 1) << a.outer_pos[b];
    return off;
}

// ------------------------------------------------------------------ tcgen05
template <int KT, int NP> struct TcCfg {
    static constexpr int TE = 1 << KT;          // complex entries per row
    static constexpr int KR = 2 * TE;           // real K = N
    static constexpr int PLANE_A = 128 * KR * 2;
    static constexpr int PLANE_B = KR * KR * 2;
    static constexpr int NPROD = NP == 1 ? 1 : NP == 2 ? 3 : 6;
    // A stages: two whole tiles when they fit next to B; else (k = 6, three
    // terms) two halves of one tile, split along K (the GEMM's column bit
    // k - 1), each accumulated in its own TMEM accumulator, so that one half
    // is converted while the other's MMAs run
    static constexpr bool WHOLE2 = (NP * PLANE_B + 2 * NP * PLANE_A) <= 200 * 1024;
    static constexpr int KH = WHOLE2 ? 1 : 2;             // K parts per tile
    static constexpr int NS = 2;                          // A stages (of a tile or of a half)
    static constexpr int SPLANE = PLANE_A / KH;           // one term plane of a stage
    static constexpr int TMEM_COLS = 2 * KH * KR;         // two accumulator sets of KH parts
    static constexpr size_t SMEM = (size_t)NP * PLANE_B + (size_t)NS * NP * SPLANE + 6144;
    // EW epilogue warps (one or two per quarter of the accumulator lanes,
    // reading all or half of the columns), 8 producer warps, 1 MMA warp. With
    // 13 warps (EW = 4) every sub-partition of the SM holds at most four, so
    // a thread may use 128 registers (the producers' register stages of a
    // tile and of an operator); 17 warps allow 96
    static constexpr int EW = 8;
    static constexpr int THREADS = 32 * (EW + 9);
    static constexpr int PROD0 = EW, MMAW = EW + 8;   // first producer warp, MMA warp
};

// Per-CTA index tables of a pass. The storage position of logical index i
// is linear over XOR in i's bits (the swizzle XORs bits 4..7 into bits 0..3),
// and the tile row, the tile column and the tile's outer bits set disjoint
// bits of i; so position = pout ^ prow[r] ^ pcol[t], and likewise the table
// index of every diagonal factor (one byte per factor, packed) =
// dout ^ drow[r] ^ dcol[t].
struct PassTables {
    int prow[128], drow[128];
    int pcol[64], dcol[64];
    int tcol[64];   // operator index of GEMM column g (its bit j is bit col_of[j] of the index)
    // the tile's 2^(k+7) entries in the producers' order: bit i of entry e
    // is tensor index bit e_bits[i] (its low 5 bits, a warp's lanes, the
    // lowest bits or nearly); tensor positions and A-operand byte offsets of
    // the low 6 and the high k + 1 bits of e (both XOR-linear in the bits)
    int plo[64], slo[64];
    int phi[128], shi[128];
};

__device__ __forceinline__ int64_t swz64(int64_t i, int swz) { return swz ? (i ^ ((i >> 4) & 15)) : i; }

__device__ __forceinline__ int diag_index_bits(const DenseArgs& a, int64_t i) {
    int e = 0;
    for (int d = 0; d < a.ndiag; ++d)
        for (int b = 0; b < a.diag_nb[d]; ++b) e |= (int)((i >> a.diag_pos[d][b]) & 1) << (8 * d + b);
    return e;
}

__device__ void fill_pass_tables(const DenseArgs& a, PassTables* T, int tid, int nthreads) {
    {
        // the entry bits with their row / column role
        int pos[13], role[13];   // role: row bit j (j), or GEMM column bit j (16 + j)
        const int nb = a.k + 7;
        for (int i = 0; i < nb; ++i) {
            pos[i] = a.e_bits[i];
            role[i] = 0;
            for (int j = 0; j < 7; ++j)
                if (a.row_pos[j] == pos[i]) role[i] = j;
            for (int j = 0; j < a.k; ++j)
                if (a.tile_pos[a.col_of[j]] == pos[i]) role[i] = 16 + j;
        }
        for (int u = tid; u < 64 + (1 << (a.k + 1)); u += nthreads) {
            const bool lo = u < 64;
            const int e = lo ? u : u - 64, b0 = lo ? 0 : 6, nbits = lo ? 6 : a.k + 1;
            int64_t off = 0;
            int rt = 0;
            for (int i = 0; i < nbits; ++i)
                if ((e >> i) & 1) {
                    off |= (int64_t)1 << pos[b0 + i];
                    const int ro = role[b0 + i];
                    rt |= ro < 16 ? 1 << ro : 1 << (8 + ro - 16);
                }
            if (lo) {
                T->plo[e] = (int)swz64(off, a.swz);
                T->slo[e] = a_offset(rt & 255, rt >> 8);
            } else {
                T->phi[e] = (int)swz64(off, a.swz);
                T->shi[e] = a_offset(rt & 255, rt >> 8);
            }
        }
    }
    for (int r = tid; r < 128; r += nthreads) {
        int64_t o = 0;
        for (int b = 0; b < 7; ++b) o |= (int64_t)((r >> b) & 1) << a.row_pos[b];
        T->prow[r] = (int)swz64(o, a.swz);
        T->drow[r] = diag_index_bits(a, o);
    }
    for (int t = tid; t < (1 << a.k); t += nthreads) {
        int64_t o = 0;
        int ti = 0;
        for (int b = 0; b < a.k; ++b) {
            o |= (int64_t)((t >> b) & 1) << a.tile_pos[a.col_of[b]];
            ti |= ((t >> b) & 1) << a.col_of[b];
        }
        T->pcol[t] = (int)swz64(o, a.swz);
        T->dcol[t] = diag_index_bits(a, o);
        T->tcol[t] = ti;
    }
}

// The diagonal factors at packed table indices e (tables of this tensor in
// shared memory, 32 entries per factor).
__device__ __forceinline__ float2 diag_product(const float2* tab, int ndiag, int e) {
    float2 f = tab[e & 31];
    for (int d = 1; d < ndiag; ++d) f = cmulf(f, tab[32 * d + ((e >> (8 * d)) & 31)]);
    return f;
}

// The deferred diagonal factors of rows a and b at this thread's NR columns
// (packed table indices da ^ dc[i], dc[i] = dcl[cs i]): per factor, the
// lookups of all 2 NR outputs are issued together, then multiplied in, so a
// shared-memory latency is paid once per factor rather than per output.
template <int NR>
__device__ __forceinline__ void row_factors(const float2* tab, int nd, int da, int db, const int* dcl, int cs,
                                            float2 (&fa)[NR], float2 (&fb)[NR]) {
    int dc[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) dc[i] = dcl[cs * i];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        fa[i] = tab[(da ^ dc[i]) & 31];
        fb[i] = tab[(db ^ dc[i]) & 31];
    }
    for (int d = 1; d < nd; ++d) {
        float2 ga[NR], gb[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            ga[i] = tab[32 * d + (((da ^ dc[i]) >> (8 * d)) & 31)];
            gb[i] = tab[32 * d + (((db ^ dc[i]) >> (8 * d)) & 31)];
        }
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            fa[i] = cmulf(fa[i], ga[i]);
            fb[i] = cmulf(fb[i], gb[i]);
        }
    }
}

template <int KT, int NP>
__global__ void __launch_bounds__(TcCfg<KT, NP>::THREADS, 1) dense_tc_kernel(const DenseArgs a) {
    using Cfg = TcCfg<KT, NP>;
    constexpr int TE = Cfg::TE, KR = Cfg::KR, KH = Cfg::KH, NS = Cfg::NS;
    constexpr int PCOLS = TE / 2;   // columns of one producer thread
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // (rounded up to 1024 bytes by pointer arithmetic on the shared array, so
    // that every pointer derived from it stays a shared-memory pointer: plain
    // shared loads and stores, which the compiler keeps apart from the global
    // ones)
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sB = smem;                                   // NP planes of B
    unsigned char* sA = smem + NP * Cfg::PLANE_B;               // NS stages x NP planes of A
    uint64_t* bars = reinterpret_cast<uint64_t*>(sA + NS * NP * Cfg::SPLANE);
    uint64_t* a_full = bars;            // [NS] producers -> MMA (256 arrivals)
    uint64_t* a_empty = bars + NS;      // [NS] MMA commit -> producers
    uint64_t* acc_full = bars + 2 * NS; // [2] MMA commit -> epilogue
    uint64_t* acc_empty = bars + 2 * NS + 2;   // [2] epilogue (32 EW arrivals) -> MMA
    int* misc = reinterpret_cast<int*>(bars + 2 * NS + 5);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(misc);     // written by tcgen05.alloc
    volatile int* abort_flag = misc + 1;                         // a bounded wait ran out
    PassTables* T = reinterpret_cast<PassTables*>(misc + 4);
    float2* stab = reinterpret_cast<float2*>(T + 1);             // [4][32] diagonal tables of the current tensor

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint64_t tiles_per = (uint64_t)1 << a.nouter;   // (dead outer legs excluded)
    const uint64_t total = a.ntens * tiles_per;
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t t_begin = (uint64_t)blockIdx.x * per;
    const uint64_t t_end = t_begin + per < total ? t_begin + per : total;
    const uint64_t N = a.stride;   // entries between consecutive tensors (>= 2^W)

    fill_pass_tables(a, T, tid, Cfg::THREADS);
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&a_full[s], 256);
            mbar_init(&a_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 32 * Cfg::EW);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == Cfg::MMAW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= Cfg::PROD0 && warp < Cfg::MMAW) {
        // ---------------------------------------------------------- producers
        // thread pt loads the tile's entries e = pt + 256 j in index order: the
        // lanes of a warp cover the tile's lowest index bits (its lowest 5,
        // which are the tensor's lowest 5 since the row bits are the lowest
        // free ones), so every warp load reads whole 128-byte lines
        const int pt = tid - 32 * Cfg::PROD0;
        constexpr int BITEMS = TE * TE / 4 / 256;   // operator chunks (4 complex entries) per thread
        uint64_t cur = ~0ull;                  // tensor whose operator is in the B planes
        for (uint64_t t = t_begin; t < t_end; ++t) {
            const uint64_t it = t - t_begin;
            const uint64_t tens = t / tiles_per, o = t % tiles_per;
            const bool newt = tens != cur;
            // positions combine by XOR (the swizzle mixes the bits of the
            // parts); the tile's loads are in flight while the previous tile's
            // MMAs still read the shared stage (a register stage in front of
            // the shared one), except after a tensor change
            const float2* src = a.L + tens * N;
            const int64_t pr = swz64(outer_offset(a, o), a.swz) ^ T->plo[pt & 63];
            const int sl = T->slo[pt & 63];
            if (newt) {
                // every MMA of the previous tile is complete before B changes;
                // then this tensor's operator goes into the B term planes (real
                // block form, K-major, 128-byte swizzle): per operator chunk
                // (row t', complex columns 4g..4g+3) the 16-byte chunks g of
                // output reals 2t' and 2t' + 1. The operator's loads are issued
                // first, in flight while those MMAs finish.
                float2 w[BITEMS][4];
                const float2* op = a.ops + tens * (uint64_t)TE * TE;
#pragma unroll
                for (int i = 0; i < BITEMS; ++i) {
                    const int u = pt + 256 * i, tp = u / (TE / 4), g = u % (TE / 4);
                    const float2* orow = op + T->tcol[tp] * TE;   // (GEMM columns in operator order)
#pragma unroll
                    for (int j = 0; j < 4; ++j) w[i][j] = orow[T->tcol[4 * g + j]];
                }
                if (it > 0) {
                    const uint64_t ul = it * KH - 1;   // the previous tile's last A unit
                    if (!mbar_wait(&a_empty[ul % NS], (uint32_t)((ul / NS) & 1), abort_flag)) break;
                }
#pragma unroll
                for (int i = 0; i < BITEMS; ++i) {
                    const int u = pt + 256 * i, tp = u / (TE / 4), g = u % (TE / 4);
#pragma unroll
                    for (int cp = 0; cp < 2; ++cp) {
                        const int n = 2 * tp + cp;
                        uint32_t h[NP][4];
#pragma unroll
                        for (int j = 0; j < 4; ++j)   // row (t', cp) of [[Re, -Im], [Im, Re]] against (t, re), (t, im)
                            pack_terms<NP>(cp == 0 ? w[i][j].x : w[i][j].y, cp == 0 ? -w[i][j].y : w[i][j].x, h, j);
                        const uint32_t off = sw128_chunk(KR, n, g >> 3, g & 7);
#pragma unroll
                        for (int qq = 0; qq < NP; ++qq)
                            *reinterpret_cast<uint4*>(sB + qq * Cfg::PLANE_B + off) =
                                make_uint4(h[qq][0], h[qq][1], h[qq][2], h[qq][3]);
                    }
                }
                cur = tens;
            }
            // the tile in KH parts (K halves: the GEMM's top column bit is the
            // top bit of j, so part h is j in [h PCOLS / KH, (h + 1) PCOLS / KH))
            bool stop = false;
#pragma unroll 1
            for (int h = 0; h < KH && !stop; ++h) {
                const uint64_t u = it * KH + h;   // A unit
                const int s = (int)(u % NS);
                unsigned char* stage = sA + (size_t)s * NP * Cfg::SPLANE;
                constexpr int PJ = PCOLS / KH;
                float2 v[PJ];
#pragma unroll
                for (int j = 0; j < PJ; ++j) v[j] = src[pr ^ T->phi[(pt >> 6) + 4 * (h * PJ + j)]];
                if (u >= (uint64_t)NS && !mbar_wait(&a_empty[s], (uint32_t)(((u / NS) - 1) & 1), abort_flag)) {
                    stop = true;
                    break;
                }
#pragma unroll
                for (int j = 0; j < PJ; ++j) {
                    uint32_t w[NP];
                    split_pair<NP>(v[j].x, v[j].y, w);
                    // (a half-tile stage holds one 64-real K block: the block bit dropped)
                    const int off = (sl ^ T->shi[(pt >> 6) + 4 * (h * PJ + j)]) & (Cfg::SPLANE - 1);
#pragma unroll
                    for (int q = 0; q < NP; ++q) *reinterpret_cast<uint32_t*>(stage + q * Cfg::SPLANE + off) = w[q];
                }
                fence_async_smem();
                mbar_arrive(&a_full[s]);
            }
            if (stop) break;
        }
    } else if (warp == Cfg::MMAW) {
        // -------------------------------------------------------------- MMA
        const uint32_t idesc = idesc_bf16(KR);
        bool stop = false;
        for (uint64_t t = t_begin; t < t_end && !stop; ++t) {
            const uint64_t it = t - t_begin;
            const int ab = (int)(it & 1);
#pragma unroll 1
            for (int h = 0; h < KH; ++h) {
                const uint64_t u = it * KH + h;
                const int s = (int)(u % NS);
                if (!mbar_wait(&a_full[s], (uint32_t)((u / NS) & 1), abort_flag)) {
                    stop = true;
                    break;
                }
                if (h == 0 && it >= 2 && !mbar_wait(&acc_empty[ab], (uint32_t)(((it >> 1) - 1) & 1), abort_flag)) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t a0 = smem_u32(sA + (size_t)s * NP * Cfg::SPLANE), b0 = smem_u32(sB);
                    const uint32_t d = tmem + (uint32_t)((ab * KH + h) * KR);   // accumulator of part h
                    int first = 1;
#pragma unroll
                    for (int pr = 0; pr < Cfg::NPROD; ++pr) {
                        // products of total order < NP, smallest first: the last three
                        // are those of NP = 2, the last one that of NP = 1
                        constexpr int PA[6] = {2, 1, 0, 1, 0, 0}, PB[6] = {0, 1, 2, 0, 1, 0};
                        constexpr int off = NP == 1 ? 5 : NP == 2 ? 3 : 0;
                        const int pa = PA[off + pr], pb = PB[off + pr];
#pragma unroll
                        for (int ks = 0; ks < KR / 16 / KH; ++ks) {
                            const int kg = h * (KR / 16 / KH) + ks;   // K step of the whole tile
                            const uint32_t koff = (uint32_t)(((ks >> 2) * 128 * 128) + (ks & 3) * 32);
                            const uint32_t kofb = (uint32_t)((kg >> 2) * KR * 128 + (kg & 3) * 32);
                            umma_bf16(d, smem_desc(a0 + pa * Cfg::SPLANE + koff),
                                      smem_desc(b0 + pb * Cfg::PLANE_B + kofb), idesc, first ? 0u : 1u);
                            first = 0;
                        }
                    }
                    umma_commit(&a_empty[s]);
                    if (h == KH - 1) umma_commit(&acc_full[ab]);
                }
                __syncwarp();
            }
        }
        // the last commits complete before tensor memory is released
        const uint64_t n = t_end > t_begin ? (t_end - t_begin) * KH : 0;
        if (n > 0) mbar_wait(&a_empty[(n - 1) % NS], (uint32_t)(((n - 1) / NS) & 1), abort_flag);
    } else {
        // --------------------------------------------------------- epilogue
        // warp w reads accumulator lanes 32 (w % 4) .. + 31 (tile rows) and
        // the columns of its halves (both, or half w / 4), 16 lanes at a time:
        // lane t holds rows t / 4 and t / 4 + 8 of the 16 at complex columns
        // t % 4 (+ 4 i), so a warp's store covers row bits 0..2 and column
        // bits 0, 1, which the host puts on the tensor's lowest index bits
        // (whole sectors)
        constexpr int EW = Cfg::EW;
        constexpr int NH = 8 / EW;          // column halves per warp
        constexpr int EC = TE / 2;          // complex columns of a half
        constexpr int NREP = EC / 4;        // 16x256b repetitions (8 real columns each)
        const int q = warp & 3, h0 = NH == 1 ? warp >> 2 : 0;
        const int rq = lane >> 2, cq = lane & 3;
        const int* pcl = T->pcol + h0 * EC + cq;   // column c of half hi: [hi * EC + 4 i]
        const int* dcl = T->dcol + h0 * EC + cq;
        uint64_t cur = ~0ull;
        for (uint64_t t = t_begin; t < t_end; ++t) {
            const uint64_t it = t - t_begin;
            const int ab = (int)(it & 1);
            const uint64_t tens = t / tiles_per, o = t % tiles_per;
            if (a.ndiag && tens != cur) {
                // this tensor's diagonal tables (the epilogue warps: named barrier 1)
                asm volatile("bar.sync 1, %0;" ::"r"(32 * EW) : "memory");
                for (int e = tid; e < a.ndiag * 32; e += 32 * EW) stab[e] = a.diag[tens * (uint64_t)a.diag_stride + e];
                asm volatile("bar.sync 1, %0;" ::"r"(32 * EW) : "memory");
                cur = tens;
            }
            if (!mbar_wait(&acc_full[ab], (uint32_t)((it >> 1) & 1), abort_flag)) break;
            tc_fence_after();
            const int64_t ob = outer_offset(a, o);
            float2* dst = a.L + tens * N;
            const int64_t pob = swz64(ob, a.swz);
            const int dob = diag_index_bits(a, ob);
            constexpr int NCH = NREP / 4;   // 16x256b.x4 loads (32 columns) per half
#pragma unroll
            for (int hi = 0; hi < NH; ++hi)
#pragma unroll
                for (int hp = 0; hp < 2; ++hp) {
                    const int r0 = 32 * q + 16 * hp + rq, r1 = r0 + 8;
                    const int64_t p0 = pob ^ T->prow[r0], p1 = pob ^ T->prow[r1];
                    float2 f0[NREP], f1[NREP];
                    if (a.ndiag)
                        row_factors<NREP>(stab, a.ndiag, dob ^ T->drow[r0], dob ^ T->drow[r1], dcl + hi * EC, 4, f0, f1);
#pragma unroll
                    for (int cc = 0; cc < NCH; ++cc) {
                        // the tile's sum: the accumulators of its KH parts
                        const uint32_t col = (uint32_t)((h0 + hi) * (KR / 2) + cc * 32);
                        const uint32_t lanes = (uint32_t)(32 * q + 16 * hp) << 16;
                        float v[16];
                        tmem_ld16x256<4>(tmem + lanes + (uint32_t)(ab * KH * KR) + col, v);
                        if constexpr (KH == 2) {
                            float w[16];
                            tmem_ld16x256<4>(tmem + lanes + (uint32_t)((ab * KH + 1) * KR) + col, w);
#pragma unroll
                            for (int j = 0; j < 16; ++j) v[j] += w[j];
                        }
                        if (hi == NH - 1 && hp == 1 && cc == NCH - 1) {
                            tc_fence_before();
                            mbar_arrive(&acc_empty[ab]);
                        }
#pragma unroll
                        for (int ii = 0; ii < 4; ++ii) {
                            const int i = 4 * cc + ii;
                            const int pc = pcl[hi * EC + 4 * i];
                            float2 y0 = make_float2(v[4 * ii], v[4 * ii + 1]);
                            float2 y1 = make_float2(v[4 * ii + 2], v[4 * ii + 3]);
                            if (a.ndiag) {
                                y0 = cmulf(y0, f0[i]);
                                y1 = cmulf(y1, f1[i]);
                            }
                            dst[p0 ^ pc] = y0;
                            dst[p1 ^ pc] = y1;
                        }
                    }
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == Cfg::MMAW) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                     : "memory");
    }
    if (tid == 0 && *abort_flag) atomicExch(a.err, 1);
}

// --------------------------------------------------------------------- SIMT
// One CTA per tile of 128 rows: the rows and the operator in shared memory,
// every thread an 8 x 4 block of complex outputs, FP32 fused multiply-adds.
template <int KT>
__global__ void __launch_bounds__(256) dense_simt_kernel(const DenseArgs a) {
    constexpr int TE = 1 << KT;
    constexpr int RB = 8, CB = TE / 16;   // rows and columns per thread (16 x 16 threads)
    extern __shared__ __align__(16) unsigned char smem_simt[];
    float2* sX = reinterpret_cast<float2*>(smem_simt);   // [TE][128]: x[row][t] at t * 128 + row
    float2* sO = sX + TE * 128;                          // [TE][TE]: Op[t'][t] at t * TE + t'
    __shared__ PassTables T;
    __shared__ float2 stab[4 * 32];
    const int tid = threadIdx.x;
    const uint64_t tiles_per = (uint64_t)1 << a.nouter;   // (dead outer legs excluded)
    const uint64_t total = a.ntens * tiles_per;
    const uint64_t N = a.stride;   // entries between consecutive tensors (>= 2^W)
    fill_pass_tables(a, &T, tid, 256);
    uint64_t cur = ~0ull;
    const int tx = tid & 15, ty = tid >> 4;
    for (uint64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const uint64_t tens = t / tiles_per, o = t % tiles_per;
        __syncthreads();
        if (tens != cur) {
            const float2* op = a.ops + tens * (uint64_t)TE * TE;
            for (int e = tid; e < TE * TE; e += 256) {
                const int tp = e / TE, ti = e % TE;   // GEMM column indices
                sO[ti * TE + tp] = op[T.tcol[tp] * TE + T.tcol[ti]];
            }
            for (int e = tid; e < a.ndiag * 32; e += 256) stab[e] = a.diag[tens * (uint64_t)a.diag_stride + e];
            cur = tens;
        }
        const int64_t ob = outer_offset(a, o);
        float2* L = a.L + tens * N;
        const int64_t pob = swz64(ob, a.swz);
        const int dob = diag_index_bits(a, ob);
        for (int e = tid; e < TE * 128; e += 256) {
            const int r = e & 127, c = e >> 7;
            sX[c * 128 + r] = L[pob ^ T.prow[r] ^ T.pcol[c]];
        }
        __syncthreads();
        float2 acc[RB][CB];
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int j = 0; j < CB; ++j) acc[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int c = 0; c < TE; ++c) {
            float2 x[RB], w[CB];
#pragma unroll
            for (int i = 0; i < RB; ++i) x[i] = sX[c * 128 + ty * RB + i];
#pragma unroll
            for (int j = 0; j < CB; ++j) w[j] = sO[c * TE + tx * CB + j];
#pragma unroll
            for (int i = 0; i < RB; ++i)
#pragma unroll
                for (int j = 0; j < CB; ++j) {
                    acc[i][j].x = fmaf(x[i].x, w[j].x, fmaf(-x[i].y, w[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(x[i].x, w[j].y, fmaf(x[i].y, w[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < RB; ++i)
#pragma unroll
            for (int j = 0; j < CB; ++j) sX[(tx * CB + j) * 128 + ty * RB + i] = acc[i][j];
        __syncthreads();
        for (int e = tid; e < TE * 128; e += 256) {
            const int r = e & 127, c = e >> 7;
            float2 y = sX[c * 128 + r];
            if (a.ndiag) y = cmulf(y, diag_product(stab, a.ndiag, dob ^ T.drow[r] ^ T.dcol[c]));
            L[pob ^ T.prow[r] ^ T.pcol[c]] = y;
        }
    }
}

int dense_fail(cudaError_t e, const char* what) {
    return set_error(PW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

std::mutex& dense_mutex() {
    static std::mutex mu;
    return mu;
}

template <int KT, int NP> int launch_tc(const DenseArgs& a, int nsm, cudaStream_t st, cudaEvent_t t0, cudaEvent_t t1) {
    using Cfg = TcCfg<KT, NP>;
    auto kern = dense_tc_kernel<KT, NP>;
    cudaError_t e;
    {
        std::lock_guard<std::mutex> lk(dense_mutex());
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    }
    if (e != cudaSuccess) return dense_fail(e, "cudaFuncSetAttribute(dense tc)");
    const uint64_t tiles = a.ntens << a.nouter;
    const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)nsm);
    if (t0) cudaEventRecord(t0, st);
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(a);
    e = cudaGetLastError();
    if (t1) cudaEventRecord(t1, st);
    return e == cudaSuccess ? PW_OK : dense_fail(e, "dense tc launch");
}

template <int KT> int launch_simt(const DenseArgs& a, int nsm, cudaStream_t st, cudaEvent_t t0, cudaEvent_t t1) {
    constexpr int TE = 1 << KT;
    const size_t smem = (size_t)(TE * 128 + TE * TE) * sizeof(float2);
    auto kern = dense_simt_kernel<KT>;
    cudaError_t e;
    {
        std::lock_guard<std::mutex> lk(dense_mutex());
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    if (e != cudaSuccess) return dense_fail(e, "cudaFuncSetAttribute(dense simt)");
    const uint64_t tiles = a.ntens << a.nouter;
    const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)nsm * 2);
    if (t0) cudaEventRecord(t0, st);
    kern<<<grid, 256, smem, st>>>(a);
    e = cudaGetLastError();
    if (t1) cudaEventRecord(t1, st);
    return e == cudaSuccess ? PW_OK : dense_fail(e, "dense simt launch");
}

}  // namespace

namespace {

// The order of the GEMM's rows and columns and of the producers' entries,
// chosen per pass from the bit roles. The producers' lanes (entry bits 0..4)
// take the tensor's lowest tile or row bits (whole sectors per warp load),
// with at least two column bits among them: the lanes' columns become the
// GEMM's lowest column bits and their rows row bits max(0, x - 2).. (x the
// lanes' columns), so that the A operand's 4-byte words written by a warp
// fall in 32 distinct banks (the 128-byte swizzle puts word (c & 3) +
// 4 ((c >> 2) ^ r) mod 8 of row r in bank order). The epilogue's lanes cover
// column bits 0, 1 and row bits 0..2: the same lowest bits.
void arrange_roles(DenseArgs& a) {
    struct Bit {
        int pos, col;   // tensor index bit; operator index bit, or -1 for a row bit
    };
    const int nb = a.k + 7;
    Bit all[13];
    for (int j = 0; j < a.k; ++j) all[j] = {a.tile_pos[j], j};
    for (int j = 0; j < 7; ++j) all[a.k + j] = {a.row_pos[j], -1};
    std::sort(all, all + nb, [](const Bit& x, const Bit& y) { return x.pos < y.pos; });
    bool lane[13] = {};
    int x = 0;
    for (int i = 0; i < 5; ++i) {
        lane[i] = true;
        x += all[i].col >= 0;
    }
    // fewer than two columns among the lowest five: the lowest (5 - y) bits
    // and the y lowest columns above them
    for (int y = 2 - x; y > 0; --y) {
        for (int i = 4; i >= 0; --i)
            if (lane[i] && all[i].col < 0) {
                lane[i] = false;
                break;
            }
        for (int i = 5; i < nb; ++i)
            if (!lane[i] && all[i].col >= 0) {
                lane[i] = true;
                break;
            }
    }
    int xl = 0;
    for (int i = 0; i < nb; ++i) xl += lane[i] && all[i].col >= 0;
    int nc = 0, ne = 0, rows[7];
    for (int j = 0; j < 7; ++j) rows[j] = -1;
    int nr = std::max(0, xl - 2);
    int top = -1;   // the last column bit (the GEMM's top one)
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < nb; ++i) {
            if (lane[i] != (pass == 0)) continue;
            if (all[i].col >= 0) {
                a.col_of[nc++] = all[i].col;
                if (nc == a.k && pass == 1) {
                    top = all[i].pos;
                    continue;   // (placed last below)
                }
            } else if (pass == 0) {
                rows[nr++] = all[i].pos;
            } else {
                int j = 0;
                while (rows[j] >= 0) ++j;
                rows[j] = all[i].pos;
            }
            a.e_bits[ne++] = all[i].pos;
        }
    // the GEMM's top column bit is the producers' top entry bit, so a K half
    // of the tile (that bit fixed) is half of every thread's entries
    if (top >= 0) a.e_bits[ne++] = top;
    for (int j = 0; j < 7; ++j) a.row_pos[j] = rows[j];
}

}  // namespace

int dense_run(int gemm, const DenseArgs& args, cudaStream_t st, cudaEvent_t t0, cudaEvent_t t1) {
    DenseArgs a = args;
    arrange_roles(a);
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    nsm = std::max(nsm, 1);
    if (a.ntens == 0) return PW_OK;
    if (gemm == PW_GEMM_FP32) return a.k == 5 ? launch_simt<5>(a, nsm, st, t0, t1) : launch_simt<6>(a, nsm, st, t0, t1);
    if (gemm == PW_GEMM_BF16)
        return a.k == 5 ? launch_tc<5, 1>(a, nsm, st, t0, t1) : launch_tc<6, 1>(a, nsm, st, t0, t1);
    if (gemm == PW_GEMM_SPLIT2)
        return a.k == 5 ? launch_tc<5, 2>(a, nsm, st, t0, t1) : launch_tc<6, 2>(a, nsm, st, t0, t1);
    return a.k == 5 ? launch_tc<5, 3>(a, nsm, st, t0, t1) : launch_tc<6, 3>(a, nsm, st, t0, t1);
}

}  // namespace pw

using namespace pw;

extern "C" int pw_dense_apply(int gemm, const pw_dense_desc* desc, uint64_t n_tensors, float* d_tensors,
                              const float* d_ops, const float* d_diag, void* stream) {
    if (!desc) return set_error(PW_ERR_ARG, "null descriptor");
    if (gemm != PW_GEMM_FP32 && gemm != PW_GEMM_BF16 && gemm != PW_GEMM_SPLIT2 && gemm != PW_GEMM_SPLIT3)
        return set_error(PW_ERR_ARG, "unknown gemm kind");
    const pw_dense_desc& d = *desc;
    if (d.tile_bits != 5 && d.tile_bits != 6) return set_error(PW_ERR_ARG, "tile_bits must be 5 or 6");
    if (d.width_bits < d.tile_bits + 7 || d.width_bits > 31)
        return set_error(PW_ERR_ARG, "width_bits must be in [tile_bits + 7, 31]");
    if (d.n_diag < 0 || d.n_diag > 4) return set_error(PW_ERR_ARG, "n_diag must be in 0..4");
    if (n_tensors && (!d_tensors || !d_ops || (d.n_diag && !d_diag))) return set_error(PW_ERR_ARG, "null buffer");
    DenseArgs a;
    std::memset(&a, 0, sizeof(a));
    a.W = d.width_bits;
    a.stride = (uint64_t)1 << a.W;
    a.k = d.tile_bits;
    a.swz = d.swizzled ? 1 : 0;
    // the tile and row bits: distinct, in range; the others are the outer bits
    uint64_t used = 0;
    auto take = [&](int b) {
        if (b < 0 || b >= a.W || ((used >> b) & 1)) return false;
        used |= 1ull << b;
        return true;
    };
    for (int j = 0; j < a.k; ++j) {
        if (!take(d.tile_pos[j])) return set_error(PW_ERR_ARG, "tile_pos: bits must be distinct and < width_bits");
        a.tile_pos[j] = d.tile_pos[j];
    }
    for (int j = 0; j < 7; ++j) {
        if (!take(d.row_pos[j])) return set_error(PW_ERR_ARG, "row_pos: bits must be distinct, < width_bits, not tile bits");
        a.row_pos[j] = d.row_pos[j];
    }
    for (int b = 0; b < a.W; ++b)
        if (!((used >> b) & 1)) a.outer_pos[a.nouter++] = b;
    a.ndiag = d.n_diag;
    a.diag_stride = 32 * d.n_diag;
    for (int i = 0; i < a.ndiag; ++i) {
        if (d.diag_bits[i] < 0 || d.diag_bits[i] > 5) return set_error(PW_ERR_ARG, "diag_bits must be in 0..5");
        a.diag_nb[i] = d.diag_bits[i];
        for (int b = 0; b < a.diag_nb[i]; ++b) {
            if (d.diag_pos[i][b] < 0 || d.diag_pos[i][b] >= a.W) return set_error(PW_ERR_ARG, "diag_pos out of range");
            a.diag_pos[i][b] = d.diag_pos[i][b];
        }
    }
    if (n_tensors == 0) return PW_OK;
    a.L = reinterpret_cast<float2*>(d_tensors);
    a.ops = reinterpret_cast<const float2*>(d_ops);
    a.diag = reinterpret_cast<const float2*>(d_diag);
    a.ntens = n_tensors;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    int* d_err = nullptr;
    if (int rc0 = dev_alloc(reinterpret_cast<void**>(&d_err), sizeof(int), "error flag")) return rc0;
    a.err = d_err;
    int rc = PW_OK;
    if ((e = cudaMemsetAsync(d_err, 0, sizeof(int), st)) != cudaSuccess) rc = dense_fail(e, "cudaMemsetAsync");
    if (!rc) rc = dense_run(gemm, a, st);
    int h_err = 0;
    if (!rc && (e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        rc = dense_fail(e, "reading the error flag");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess && !rc) rc = dense_fail(e, "cudaStreamSynchronize");
    dev_free(d_err);
    if (!rc && h_err) rc = set_error(PW_ERR_TIMEOUT, "a bounded wait of the tensor-core pass ran out");
    return rc;
}

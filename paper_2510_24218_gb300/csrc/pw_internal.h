// Internal structures shared by the circuit builder, the planner and the CUDA
// sampler. Host-only parts are guarded so the header also compiles in .cu files.
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pw.h"

namespace pw {

using cd = std::complex<double>;

// ----------------------------------------------------------------- errors
int set_error(int code, const std::string& msg);

// ------------------------------------------------------- device memory
// Internal device buffers: the registered allocator (pw_set_allocator) or
// cudaMalloc; dev_free releases through the pair that allocated.
int dev_alloc(void** out, size_t bytes, const char* what);
void dev_free(void* p);

// ---------------------------------------------------------------- circuit
enum OpKind { OP_GATE = 0, OP_KRAUS = 1 };

struct Op {
    int kind = OP_GATE;
    std::vector<int> qubits;
    int k = 1;                 // number of matrices (Kraus operators)
    std::vector<cd> mats;      // k matrices of dim x dim, row-major
    int dim() const { return 1 << (int)qubits.size(); }
    const cd* mat(int i) const { return mats.data() + (size_t)i * dim() * dim(); }
};

bool is_diagonal(const cd* A, int dim);
bool is_monomial(const cd* A, int dim);

}  // namespace pw

struct pw_circuit {
    int n = 0;
    std::vector<pw::Op> ops;
};

namespace pw {

// ------------------------------------------------------ device plan layout
// Micro-op kinds applied to a chain's frontier tensor (2^W complex values).
enum MicroKind : uint8_t {
    MK_MAT1 = 0,   // 2x2 matrix on one bit: out[a'] = sum_a M[a'][a] in[a]
    MK_DIAG = 1,   // multiply by table[bits gathered from the index]
    MK_CONST = 2,  // multiply by one scalar
};

// How the micro-op's matrix / table is built for a given chain.
enum Recipe : uint8_t {
    RC_EXPAND = 0,      // M = [[1,0],[1,0]]: a new leg, constant along it
    RC_SUMOUT1 = 1,     // M = [[1,1],[0,0]]: sum a leg out
    RC_SUMOUT_MIX = 2,  // M = [[w0,w1],[0,0]], w = A'_{layer,qa}[s_qa][.]
    RC_REPLACE = 3,     // M[a'][a] = prod_g D'_g(qa<-a, qb<-a') * (layer>=0 ? A'_{layer,qa}[s_qa][a] : 1)
    RC_BREPLACE = 4,    // M[a][a'] = prod_g D'_g(qa<-a, qb<-a')   (in: qb's leg, out: qa's leg)
    RC_EDGE = 5,        // table[a + 2b] = prod_g D'_g(qa<-a, qb<-b)
    RC_SITE = 6,        // site tensor of qa over its open segments (see sampler)
    RC_CONST_EDGES = 7, // prod_g D'_g(s_q0, s_q1)
};

struct DevMicroOp {
    uint8_t kind;
    uint8_t recipe;
    uint8_t nbits;
    uint8_t fixed_top;   // RC_SITE: top segment fixed to s (backward sweep)
    uint8_t bits[4];
    uint8_t fpos[4];     // positions of bits[] inside the fused op's diagonal bits
    int16_t qa, qb;
    int16_t layer;       // mixer layer of the top weight (-1: none); RC_SITE: number of segments
    int16_t pad0;
    int32_t glist;       // first index into gate_refs
    int32_t gcount;
};

// A tiled pass: every thread loads tiles of 2^ntb entries (the index bits
// tbits[] varying, the others fixed), runs the pass's stages on them in
// registers and stores them back. A stage is a 2x2 matrix on one tile bit, or
// a diagonal factor over up to 5 bits (tile bits or fixed bits), the product
// of consecutive diagonal/scalar micro-ops.
enum StageType : uint8_t { ST_MAT = 0, ST_DIAG = 1 };
// Shape of a 2x2 stage's matrix M[out][in], known from its micro-op: general;
// expand (M = c [[1,0],[1,0]], c real: 1, or the program's pending power of
// two when it is the first stage); row 0 (M = [[w0,w1],[0,0]]).
enum MatForm : uint8_t { MF_GENERAL = 0, MF_EXPAND = 1, MF_ROW0 = 2 };
struct DevStage {
    uint8_t type;
    uint8_t arg;         // ST_MAT: index into tbits; ST_DIAG: number of diagonal bits
    uint8_t dbits[5];    // ST_DIAG: index bits of the table, entry bit j <- index bit dbits[j]
    uint8_t tpos[4];     // ST_DIAG: position in dbits of tile bit k, 0xFF if absent
    uint8_t ndep;        // precomputed table: chain bits it depends on (0..4); 0xFF: built at run time
    uint8_t form;        // ST_MAT: MatForm
    uint8_t epi;         // dense pass: a diagonal factor applied after the pass's operator
    int32_t op_begin, op_end;   // constituent micro-ops
    int32_t tab_off;            // complex entries from the start of the block's table area
    int16_t dep[4];             // qubits whose current bits select the variant
    int32_t var_off;            // first entry of variant 0 in the precomputed tables
};
struct DevFused {
    uint8_t ntb;         // tile bits (0..4; a dense pass: 5 or 6)
    uint8_t tbits[8];
    uint8_t nst;         // stages (1..8; a dense pass: any number)
    uint8_t pad[2];
    int32_t st_begin;    // first DevStage
};

// A diagonal cost gate (1 or 2 qubits) with its table; level = segment index.
// The kernel loads d[] as double2 and f[] as float2: d must start on a 16-byte
// boundary and the struct size must keep that true along an array.
struct alignas(16) DevCostGate {
    double d[8];         // 4 complex (re, im) entries, local index b0 + 2 b1
    float f[8];          // the same in FP32
    int16_t q0, q1;      // q1 < 0 for a one-qubit gate
    int16_t level;
    int16_t pad;
};
static_assert(offsetof(DevCostGate, d) % 16 == 0 && offsetof(DevCostGate, f) % 8 == 0, "vector loads");
static_assert(sizeof(DevCostGate) % 16 == 0, "array stride keeps d aligned");

// Items of a cost section. Within a section they are grouped into waves: the
// items of one wave touch disjoint frame bits and one-qubit factors, so the
// kernel runs a wave in parallel; waves run in order, and every item comes
// after the items it depends on (same result as circuit order).
enum CostItemKind : int16_t { CI_GATE2 = 0, CI_GATE1 = 1, CI_CHANNEL = 2 };
struct DevCostItem {
    int16_t kind;
    int16_t pad;
    int32_t idx;         // cost gate index or channel index
};

struct DevKrausFactor {
    int16_t q;
    int16_t antidiag;    // 1: factor is anti-diagonal, flips the frame bit
    int32_t pad;
    double d[4];         // diagonal (after the sigma_X fold) as (re, im) x 2
};

struct DevChannel {
    int32_t op_id;
    int16_t nq, k;
    int16_t q[2];
    int32_t cum_off;     // [2^nq][k] cumulative probabilities (FP64)
    int32_t fac_off;     // [k][nq] factors
};

// A site resampled in a readout block.
struct DevBlockSite {
    int16_t q;
    int16_t monomial;    // 1: deterministic move
    int32_t op_id;
    int32_t trace_row;   // -1 when the update is deterministic
    int32_t pad;
};

// A live frontier slot at a readout.
struct DevLiveSlot {
    int16_t q;           // qubit, -1 if the slot is free
    int16_t role;        // index of the site inside the block, or -1 (done earlier)
    int32_t dlist;       // gate refs of the cross edges to unabsorbed qubits
    int32_t dcount;
    int16_t ndep;        // precomputed factor: chain bits it depends on; 0xFF: run time
    int16_t dep[5];
    int32_t var_off;     // 2 entries per variant in the precomputed tables
};

// Per (layer m >= 1, block k) ranges.
struct DevBlockRange {
    int32_t fwd_begin, fwd_end;     // DevFused of the forward absorption of block k
    int32_t bwd_begin, bwd_end;     // DevFused turning R_k into R_{k-1}
    int32_t site_begin, site_end;   // DevBlockSite
    int32_t live_begin, live_end;   // DevLiveSlot
    int32_t fwd_tab, bwd_tab;       // table entries of the two programs
    int32_t fwd_st, bwd_st;         // first stage of the two programs
    int32_t fwd_nst, bwd_nst;       // their stage counts
    int32_t rmask;                  // slots holding the block's sites
    int8_t rslot[12];               // slot of the i-th site of the block
};

struct DevPlanHeader {
    int32_t n, P;              // qubits, mixer layers after the first
    int32_t S;                 // slots
    int32_t K;                 // blocks
    int32_t n_ops;
    int32_t n_cost_gates;
    int32_t n_channels;
    int32_t n_sampled;         // trace rows
    int32_t max_block;
    int32_t has_segfac;        // 1-qubit diagonal gates or channels present
    int32_t has_frame;         // channels present
    int32_t words;             // uint64 words per bitstring
    int32_t max_tab;           // max table entries of one block program
    int32_t max_stages;        // max stages of one block program
    int32_t clean_tables;      // noisy plan whose variant tables assume Kraus pick 0 everywhere
    int32_t amp_exp;           // power of two of every amplitude left out of the tables
    int32_t dense_mask;        // bit m: layer m's forward passes are dense GEMM passes (HBM frontier)
    int32_t dense_npass;       // most dense passes of one forward block program
};

// Offsets (in bytes) of the arrays inside the device blob.
struct DevPlanOffsets {
    int64_t micro, fused, stages, row_opid, vtab_f, vtab_d, gate_refs, cost_gates, cost_items, cost_ranges, cost_waves, cost_wave_ranges, channels, cum,
        factors;
    int64_t mix_d, mix_f, mix0_order, mix0_opid, mix_mono, segdef_d, segdef_f;
    int64_t block_ranges, block_sites, live_slots;
};

}  // namespace pw

#ifndef __CUDACC__
#endif

struct pw_plan_host;  // forward

namespace pw {

struct HostPlan {
    DevPlanHeader hdr{};
    // blob pieces (host copies)
    std::vector<DevMicroOp> micro;
    std::vector<DevFused> fused;
    std::vector<DevStage> stages;
    std::vector<int32_t> row_opid;        // op id of each sampled gate (trace row)
    std::vector<float> vtab_f;            // precomputed stage / slot tables (complex), FP32
    std::vector<double> vtab_d;           // the same in FP64
    std::vector<int32_t> gate_refs;
    std::vector<DevCostGate> cost_gates;
    std::vector<DevCostItem> cost_items;
    std::vector<int32_t> cost_ranges;      // [P+2]: items of section m in [r[m], r[m+1]) (m = 1..P+1 used)
    std::vector<int32_t> cost_waves;       // first item of every wave, then the item count
    std::vector<int32_t> cost_wave_ranges; // [P+3]: waves of section m in [w[m], w[m+1])
    std::vector<DevChannel> channels;
    std::vector<double> cum;
    std::vector<DevKrausFactor> factors;
    std::vector<double> mix_d;             // [(P+1) * n * 8]  (2x2 complex, [o][i])
    std::vector<float> mix_f;
    std::vector<int32_t> mix0_order;       // qubits of mixer layer 0 in circuit order
    std::vector<int32_t> mix0_opid;        // op id of mixer-0 gate per qubit
    std::vector<int8_t> mix_mono;          // [(P+1) * n]: 1 if the mixer is monomial
    std::vector<double> segdef_d;          // [n][P+1][2] complex: segment factors of a clean chain
    std::vector<float> segdef_f;
    std::vector<DevBlockRange> block_ranges;   // [(P+1) * K] (layer 0 unused)
    std::vector<DevBlockSite> block_sites;
    std::vector<DevLiveSlot> live_slots;

    std::vector<int> exec_order;          // op ids in execution order
    std::vector<int> sweep_order;         // qubit order pi
    std::vector<std::vector<int>> blocks; // qubits per block
    int W = 0, W_low = 0;                 // at the deepest layer
    double flops_per_sample = 0.0;
    double amps_per_sample = 0.0;
    double flops_per_amplitude = 0.0;   // pw_amplitudes of the whole circuit
    int precision = PW_PREC_FP32;
    int threads_per_chain = 0;
    int chains_per_cta = 1;
    int chains_per_launch = 0;
    int ctas_per_chain = 1;               // > 1: one thread-block cluster per chain
    int engine = 0;                       // 1: the frontier lives in HBM, dense layers run GEMM passes
    int gemm = PW_GEMM_SPLIT3;            // arithmetic of the dense passes
    int dense_k = 0;                      // tile bits of the widest dense layer's passes
    double dense_flops_per_sample = 0.0;  // real flops of the dense passes (dense operators) per sample
    double dense_passes_per_sample = 0.0;
    // dense passes (by fused index): the frontier bits that may be nonzero
    // before and after the pass (a summed-out leg is zero until a new site
    // expands it; the frontier starts as a delta at index 0)
    std::vector<uint32_t> pass_live_in, pass_live_out;
    int wloc = 0;                         // log2 of the frontier entries per CTA then
    size_t smem_per_chain = 0;
    bool noisy = false;
    // amplitude API helpers: position of every executed mixer op (layer, block, index)
    std::vector<int> exec_layer, exec_block, exec_pos;
};

// Index bits of dense pass fi on a 2^W frontier: its tile bits, the 7 row
// bits of a GEMM tile (the lowest live bits outside the tile, then dead ones
// if too few are live) and the outer bits the tiles enumerate (the other live
// bits: a tile with a dead leg set holds zeros before and after the pass and
// is skipped). Returns the number of outer bits.
inline int dense_pass_bits(const HostPlan& hp, int fi, int W, int* rows, int* outer) {
    const DevFused& f = hp.fused[fi];
    uint32_t tb = 0;
    for (int j = 0; j < f.ntb; ++j) tb |= 1u << f.tbits[j];
    const uint32_t live = hp.pass_live_in.empty() ? ~0u : hp.pass_live_in[fi];
    int nr = 0, no = 0;
    for (int pass = 0; pass < 2; ++pass)   // live bits first, then dead ones for the rows
        for (int b = 0; b < W && nr < 7; ++b) {
            const bool l = (live >> b) & 1;
            if (((tb >> b) & 1) || l != (pass == 0)) continue;
            rows[nr++] = b;
            tb |= 1u << b;
        }
    for (int b = 0; b < W; ++b)
        if (!((tb >> b) & 1) && ((live >> b) & 1)) outer[no++] = b;
    return no;
}

int build_plan(const pw_circuit* c, const pw_plan_opts& opts, HostPlan& out);
size_t plan_device_bytes(const HostPlan& hp);

}  // namespace pw

struct pw_plan {
    pw::HostPlan hp;
    // device side (lazily created on first use)
    int device = -1;
    void* d_blob = nullptr;
    size_t blob_bytes = 0;
    pw::DevPlanOffsets off{};
    unsigned long long* d_counters = nullptr;
    void* d_stage = nullptr;       // staging for pw_sample_host
    size_t stage_bytes = 0;
    // SWAP-class gates are planned as relabellings of the qubit wires: output
    // bit q is the bit of wire out_wire[q] (empty: the identity)
    std::vector<int> out_wire;
    int* d_out_wire = nullptr;
    int* d_in_wire = nullptr;   // the inverse map: wire w holds qubit d_in_wire[w]
    // HBM engine (hp.engine == 1): frontiers, environments, saved chain states,
    // dense operators, operator images, error flag, for dense_chains chains
    void* d_dense = nullptr;
    size_t dense_bytes = 0;
    uint64_t dense_chains = 0;
    std::vector<void*> dense_events;   // cudaEvent_t pairs timing the dense passes of a call
};

namespace pw {
// Reorder the packed output rows of a plan with relabelled wires in place
// (stream: a cudaStream_t).
int permute_output(pw_plan* plan, uint64_t* d_bits, uint64_t n_samples, void* stream);
// Copy qubit-ordered packed rows to wire order (dst: n_strings rows).
int permute_input(pw_plan* plan, const uint64_t* d_src, uint64_t* d_dst, uint64_t n_strings, void* stream);
}  // namespace pw

/*
 * pw.h - C ABI of the GB300 pilot-wave exact sampler.
 *
 * The library samples bitstrings exactly from the output distribution of a
 * circuit U_T ... U_1 |0^n> with the gate-by-gate Markov chain of
 * Kalachev et al., "Pilot-Wave Simulator" (arXiv 2510.24218):
 *   - Sec. 2, Eq. (1) and Alg. 1: a classical state s is carried through the
 *     circuit; monomial gates move it deterministically, other gates resample
 *     it inside the gate's block with probability |amp(C_t,y)|^2 / sum_block,
 *     amp(C_t,i) = <i|C_t|0^n> being a tensor-network contraction;
 *   - Sec. 3 and Alg. 2 (App. A): noise channels with local-submonomial (LSM)
 *     Kraus operators are sampled by Eq. (5) and handled by X-frame propagation,
 *     so the noisy network keeps the noiseless shape (Prop. 2).
 *
 * All calls return 0 (PW_OK) or a negative PW_ERR_* code; pw_last_error()
 * returns a thread-local message for the last failure. No exception crosses
 * the ABI. Handles (pw_circuit, pw_plan) are owned by the library and freed by
 * the matching *_destroy call. Device buffers passed in are owned by the
 * caller; the library never frees them. Host arrays are read during the call
 * only.
 *
 * Conventions (the paper leaves these open):
 *   - qubit q <-> bit (q % 64) of 64-bit word (q / 64) in packed bitstrings;
 *   - an m-qubit matrix acting on (q_0..q_{m-1}) is indexed by
 *     sum_i b(q_i) 2^i (q_0 least significant), row-major, complex numbers as
 *     interleaved (re, im) doubles;
 *   - randomness: u = Philox4x32-10(key = seed, counter = (sample id, op id,
 *     purpose)) mapped to a 53-bit double; UpdateState picks the smallest
 *     candidate y (ascending local index) with u*P < sum_{y'<=y} p_{y'}, the
 *     Kraus draw applies the same rule over the Kraus list order, with Eq. (5)
 *     evaluated at the true bit s XOR x. Sample k depends only on
 *     (seed, k, circuit, plan order), so disjoint sample ranges can be run
 *     anywhere and concatenated.
 */
#ifndef PW_H
#define PW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PW_OK 0
#define PW_ERR_ARG (-1)          /* invalid argument (null, range, shape) */
#define PW_ERR_NOT_LSM (-2)      /* Kraus operator not local-submonomial (App. A) */
#define PW_ERR_OOM (-3)          /* host or device allocation failed */
#define PW_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define PW_ERR_TIMEOUT (-5)      /* reserved: a bounded device wait ran out */
#define PW_ERR_NUMERIC (-6)      /* non-finite value in inputs or results */
#define PW_ERR_UNSUPPORTED (-7)  /* circuit outside the supported structure */
#define PW_ERR_TOO_LARGE (-8)    /* plan does not fit the device limits */

#define PW_PREC_FP32 0           /* contraction in FP32, conditionals in FP64 */
#define PW_PREC_FP64 1           /* contraction and conditionals in FP64 */

#define PW_ORDER_AUTO 0          /* search sweep orders, keep the narrowest */
#define PW_ORDER_NATURAL 1       /* sweep qubits in index order */

#define PW_ENGINE_AUTO 0         /* on-chip frontier when it fits, else the HBM engine */
#define PW_ENGINE_ONCHIP 1       /* frontier in shared memory (one CTA or a cluster per chain) */
#define PW_ENGINE_HBM 2          /* frontier in HBM; wide layers' passes are dense GEMMs */

/* Arithmetic of a dense pass (pw_dense_apply, and the HBM engine's passes). */
#define PW_GEMM_SPLIT3 0   /* tensor cores: operands split into three BF16 terms (the 24-bit
                              FP32 significand), 6 products, FP32 accumulation (the default) */
#define PW_GEMM_SPLIT2 1   /* tensor cores: two BF16 terms (16 bits), 3 products */
#define PW_GEMM_BF16 2     /* tensor cores: BF16 operands (one term) */
#define PW_GEMM_FP32 3     /* FP32 CUDA cores (SIMT), the plain-FP32 arm */

typedef struct pw_circuit pw_circuit;
typedef struct pw_plan pw_plan;

/* Options of pw_plan_build. Zero-initialise for defaults. */
typedef struct {
    int precision;          /* PW_PREC_FP32 (default) or PW_PREC_FP64 */
    int order;              /* PW_ORDER_AUTO (default) or PW_ORDER_NATURAL */
    int max_block;          /* max sites resampled per readout block; 0 -> 8 */
    int threads_per_chain;  /* CUDA threads cooperating on one chain (per CTA of a cluster);
                               0 -> auto (32..256, 512 per CTA of a cluster); else a power
                               of two in 32..256 */
    int chains_per_launch;  /* chains per kernel launch; 0 -> all requested samples */
    int ctas_per_chain;     /* 0 -> auto (a thread-block cluster only when one CTA's
                               shared memory cannot hold the frontier); 2, 4 or 8
                               force that split of the frontier over a cluster */
    int engine;             /* PW_ENGINE_AUTO (default): the on-chip engine, or the HBM
                               engine when the frontier exceeds 2^17 entries (FP32 plans);
                               PW_ENGINE_HBM forces the HBM engine (FP32 plans only) */
    int gemm;               /* HBM engine: arithmetic of the dense passes, PW_GEMM_*
                               (default PW_GEMM_SPLIT3: tensor cores at FP32-equivalent
                               input precision) */
    int reserved[4];
} pw_plan_opts;

/* Shape and cost of a plan (pw_plan_stats). */
typedef struct {
    int n_qubits;
    int n_ops;              /* operations of the circuit (gates + channels) */
    int n_layers;           /* mixer layers after the first one (QAOA depth p) */
    int n_slots;            /* frontier sites kept by the sweep */
    int width_bits;         /* log2 of the frontier tensor at the deepest layer */
    int width_low_bits;     /* log2 of the cached right environments */
    int n_blocks;           /* readout blocks per layer */
    int sampled_gates;      /* non-monomial gates whose update needs amplitudes
                               (excluding the first mixer layer, which acts on a
                               product state); rows of the amplitude trace */
    int threads_per_chain;
    int chains_per_cta;
    int smem_bytes_per_cta;
    int noisy;              /* 1 if the circuit has Kraus channels */
    double flops_per_sample;   /* real flops of the contraction per sample */
    double amps_per_sample;    /* amplitudes evaluated per sample */
    double device_bytes;       /* bytes of plan tables copied to the device on first use */
    int ctas_per_chain;        /* > 1: one chain per thread-block cluster of that many CTAs */
    double flops_per_amplitude;   /* real flops of pw_amplitudes of the whole circuit, per string */
    int engine;                /* PW_ENGINE_ONCHIP or PW_ENGINE_HBM */
    int gemm;                  /* HBM engine: PW_GEMM_* of its dense passes */
    int dense_tile_bits;       /* HBM engine: tile bits k of the widest layer's dense passes */
    double dense_passes_per_sample;   /* HBM engine: dense GEMM passes per chain */
    double dense_flops_per_sample;    /* HBM engine: real flops of those passes per chain
                                         (2^W x 2^k complex multiply-adds each, 8 flops) */
} pw_plan_stats_t;

/* Counters of one pw_sample call. */
typedef struct {
    uint64_t near_boundary;   /* draws with |u*P - cum| < 1e-6 P */
    uint64_t zero_mass;       /* updates whose block had zero probability */
    uint64_t launches;        /* kernel launches issued */
    /* HBM engine (measured only when the call gets a stats pointer): */
    uint64_t dense_passes;    /* dense GEMM passes launched */
    double dense_ms;          /* their GEMM kernels' total device time (CUDA events around each) */
    double dense_bytes;       /* their algorithmic HBM bytes: every tensor entry read and
                                 written once, 16 bytes per complex FP32 entry */
    double dense_flops;       /* their dense flops: 2^W x 2^k complex multiply-adds (8 flops)
                                 per chain, times the products of the split (1, 3 or 6) */
} pw_run_stats_t;

/* ---------------------------------------------------------------- circuit */

/* New empty circuit on n_qubits (1..4096). */
int pw_circuit_create(int n_qubits, pw_circuit** out);

/* Append a gate (A, q) (App. A): m = 1 or 2 qubits, A = 2^m x 2^m complex
 * matrix, row-major, interleaved (re, im). Unitarity is not checked. */
int pw_circuit_add_gate(pw_circuit* c, int m, const int* qubits, const double* A);

/* Append a noise operation with k Kraus operators E_0..E_{k-1} (Sec. 3.1),
 * each 2^m x 2^m as in pw_circuit_add_gate, stored one after the other.
 * Every E_i must be a tensor product of 2x2 matrices with at most one nonzero
 * per row and column (LSM, App. A), else PW_ERR_NOT_LSM. The list order is the
 * order of the Kraus draw. */
int pw_circuit_add_kraus(pw_circuit* c, int m, const int* qubits, int k, const double* E);

/* The QAOA circuit of App. D on n qubits: H on every qubit; for l = 0..p-1:
 * RZZ(2 gammas[l] w[e]) = exp(-i gammas[l] w[e] Z_u Z_v) on every edge
 * (edges = 2*n_edges ints, pairs u != v) in list order, each followed by the
 * two-qubit depolarizing channel (1-depol2) rho + depol2/15 sum_{P != II} P rho P
 * when depol2 > 0 (Kraus index a + 4b: Pauli a (I,X,Y,Z) on u, Pauli b on v);
 * RZ(2 gammas[l] h[j]) on every qubit when h != NULL; RX(2 betas[l]) on qubits
 * 0..n-1; then amplitude damping E0 = diag(1, sqrt(1-g)), E1 = sqrt(g)|0><1|
 * with g = ad_gamma on qubits 0..n-1 when ad_gamma > 0. */
int pw_circuit_qaoa(int n, int n_edges, const int* edges, const double* w, const double* h,
                    int p, const double* gammas, const double* betas,
                    double depol2, double ad_gamma, pw_circuit** out);

/* Number of operations appended so far. */
int pw_circuit_num_ops(const pw_circuit* c, int* n_ops);

void pw_circuit_destroy(pw_circuit* c);

/* ------------------------------------------------------------------- plan */

/* Build the contraction plan (host only, no CUDA call). Supported structure:
 * layers of one non-diagonal 1-qubit gate per qubit (the first acting on
 * |0^n>), separated by sections of diagonal 1- or 2-qubit gates and LSM
 * channels; channels may also follow the last layer. A diagonal gate or
 * channel placed inside a layer is accepted when it commutes out of it: all
 * its qubits already had their gate of that layer (it moves after the layer)
 * or none did (it moves before). A two-qubit gate of the form SWAP x diagonal
 * (exact zero pattern: SWAP, iSWAP, fSim(pi/2, phi)) is accepted in noiseless
 * circuits: it exchanges two qubits' contents (a deterministic move, Alg. 1),
 * planned by relabelling the qubit wires, with the output bits permuted back;
 * for such plans pw_amplitudes takes only the whole circuit (it then also
 * allocates a reordered copy of the strings and synchronises the stream) and
 * pw_sample_static refuses them (PW_ERR_UNSUPPORTED).
 * Anything else returns PW_ERR_UNSUPPORTED.
 * The plan fixes the order of the commuting one-qubit gates inside each layer
 * and of the moved operations (see pw_plan_exec_order). */
int pw_plan_build(const pw_circuit* c, const pw_plan_opts* opts, pw_plan** out);

int pw_plan_stats(const pw_plan* plan, pw_plan_stats_t* out);

/* The execution order used by the plan: order[t] is the index (in insertion
 * order) of the t-th operation executed. order has n_ops entries. */
int pw_plan_exec_order(const pw_plan* plan, int* order);

void pw_plan_destroy(pw_plan* plan);

/* ------------------------------------------------------------- execution */

/* Draw samples first_sample .. first_sample + n_samples - 1 (Alg. 1 / Alg. 2).
 * d_out_bits: device buffer of n_samples * ceil(n/64) uint64 (packed s XOR x).
 * d_trace (nullable): device buffer of n_samples * sampled_gates * 4 doubles;
 *   row r of sample k holds (re, im) of amp(C_t, y) for y = 0, 1 of the r-th
 *   sampled gate, where C_t is the executed prefix including that gate.
 * stream: a cudaStream_t (NULL = legacy default stream). The call is
 * asynchronous with respect to the host unless stats != NULL, in which case it
 * synchronises the stream to read the counters. The first call of a plan on a
 * device uploads its tables (synchronously), and on the HBM engine allocates
 * its buffers; later calls with stats == NULL only enqueue work on the
 * stream. For on-chip engine plans such a call can be captured into a CUDA
 * graph (a test replays one). */
int pw_sample(pw_plan* plan, uint64_t seed, uint64_t first_sample, uint64_t n_samples,
              uint64_t* d_out_bits, double* d_trace, void* stream, pw_run_stats_t* stats);

/* Tune the plan's launch shape on this device (not in the paper: a runtime
 * choice). Times sampling trial_samples chains (0: four times the plan's
 * chains per launch, 4096 if unset; fastest of three calls after a warm-up)
 * for every threads-per-chain value in 32..256 and keeps the fastest in the
 * plan; *chosen (nullable) gets it.
 * Plans on a thread-block cluster keep their shape. The sampled bits do not
 * depend on the choice (counter-based draws), only the rounding of the
 * amplitudes may. Allocates and frees a scratch output of trial_samples
 * words per chain, synchronises the stream; returns PW_ERR_CUDA when no
 * configuration runs. */
int pw_plan_autotune(pw_plan* plan, uint64_t trial_samples, void* stream, int* chosen);

/* Plan-shape search for a circuit (the schedule, not the arithmetic): builds
 * and times plans of c over the options that change only how the sampler
 * runs - engine (FP32 plans), max_block, order, threads_per_chain,
 * chains_per_launch - one dimension at a time from *base (nullable: defaults),
 * each shape timed as the fastest of two pw_sample calls of trial_samples
 * chains (0: 16384) after a warm-up on `stream`, and writes the fastest
 * options to *best (its rate, samples/s, to *samples_per_s, nullable).
 * Fields of *base that are nonzero stay as given; precision and gemm are
 * never changed. Sweep order changes which chain a seed draws (the order of
 * commuting mixer gates), not the distribution; the other options change
 * only the rounding of amplitudes.
 * cache_path (nullable): a JSON-lines file, one object per tuned circuit
 * {"key", "device", "engine", "max_block", "order", "threads_per_chain",
 * "chains_per_launch", "samples_per_s"}; the key hashes the circuit (qubits,
 * matrices) and *base, the device names the GPU model and SM count. A matching line is returned without timing (*from_cache = 1); a new
 * result is appended (PW_ERR_ARG if the file cannot be written). Allocates a
 * scratch output of trial_samples words per chain and synchronises the
 * stream. */
int pw_autotune(const pw_circuit* c, const pw_plan_opts* base, uint64_t trial_samples, const char* cache_path,
                void* stream, pw_plan_opts* best, double* samples_per_s, int* from_cache);

/* The same with HOST buffers: h_out_bits (n_samples * ceil(n/64) uint64) and
 * the optional h_trace are written before return; device staging memory is
 * held by the plan and reused between calls. */
int pw_sample_host(pw_plan* plan, uint64_t seed, uint64_t first_sample, uint64_t n_samples,
                   uint64_t* h_out_bits, double* h_trace, pw_run_stats_t* stats);

/* amp(C_t, x) = <x|C_t|0^n> (Sec. 2) for n_strings bitstrings x (device,
 * packed like pw_sample's output), where C_t is the executed prefix of length
 * prefix_ops (pw_plan_exec_order); the prefix must end right after a
 * one-qubit mixer gate of a layer >= 1 and the circuit must be noiseless.
 * d_amp: device buffer of 2 * n_strings doubles (re, im). */
int pw_amplitudes(pw_plan* plan, int prefix_ops, uint64_t n_strings, const uint64_t* d_bits,
                  double* d_amp, void* stream);

/* Derivatives of QAOA amplitudes with respect to the angles (not in the
 * paper: an interface of this library built on the amplitude contraction of
 * Sec. 2). For the noiseless circuit of pw_circuit_qaoa with the same
 * arguments, writes, for each of the n_strings bitstrings x (device, packed
 * like pw_sample's output):
 *   d_amp  (nullable, device): 2 * n_strings doubles, amp(C, x) as (re, im);
 *   d_grad (device): n_strings * 2p * 2 doubles; row k holds
 *          d amp / d gammas[0..p-1] then d amp / d betas[0..p-1], each (re, im).
 * Exact (parameter-shift rule): every angle enters through gates exp(-i t G)
 * with G^2 = I, and d/dt exp(-i t G) = exp(-i (t + pi/2) G); each derivative is
 * the weighted sum of the amplitudes of circuits with one gate advanced by a
 * quarter turn, i.e. p(n_edges + n) contractions, plus p*n with fields h.
 * opts: the plan options used for every contraction (precision, order, ...).
 * Allocates and frees plans and an n_strings scratch vector; synchronises the
 * stream before it returns. Errors of pw_plan_build / pw_amplitudes are
 * passed on (a circuit the planner cannot take returns PW_ERR_UNSUPPORTED
 * before any device work); p < 1 returns PW_ERR_ARG. */
int pw_qaoa_amp_grad(int n, int n_edges, const int* edges, const double* w, const double* h, int p,
                     const double* gammas, const double* betas, const pw_plan_opts* opts,
                     uint64_t n_strings, const uint64_t* d_bits, double* d_amp, double* d_grad, void* stream);

/* Derivatives of amplitudes of a parameterised noiseless circuit (not in the
 * paper; built on the amplitude contraction of Sec. 2). Operation i of c
 * depends on parameter param_of_op[i] in 0..n_params-1, or on none (-1);
 * param_of_op has one entry per operation (pw_circuit_num_ops). dmats holds,
 * for every operation with a parameter, in operation order, the derivative of
 * its matrix with respect to that parameter (2^m x 2^m complex, row-major,
 * interleaved (re, im), as in pw_circuit_add_gate). By the product rule
 *   d amp(x) / d theta_k = sum over operations i with param_of_op[i] = k of
 *                          amp(c with operation i's matrix replaced by dmats_i, x);
 * each replaced circuit must still be one the planner accepts (a diagonal gate
 * with a diagonal derivative, a one-qubit gate with a one-qubit derivative),
 * else the planner's error is returned. Writes d_amp (nullable, device,
 * 2 * n_strings doubles: amp(c, x)) and d_grad (device, n_strings * n_params * 2
 * doubles; row k holds d amp / d theta_0..n_params-1, each (re, im)); a
 * parameter no operation depends on gets zeros. Bitstrings d_bits as in
 * pw_amplitudes. Exact up to rounding; the rows are deterministic. Allocates
 * and frees plans and scratch, synchronises the stream before it returns.
 * Errors: PW_ERR_ARG (null pointers, n_params < 1, an entry out of range, a
 * channel with a parameter), PW_ERR_NUMERIC (non-finite derivative entry),
 * and those of pw_plan_build / pw_amplitudes (a noisy circuit is
 * PW_ERR_UNSUPPORTED). */
int pw_amp_grad(const pw_circuit* c, int n_params, const int* param_of_op, const double* dmats,
                const pw_plan_opts* opts, uint64_t n_strings, const uint64_t* d_bits, double* d_amp,
                double* d_grad, void* stream);

/* Score-function estimate of the gradient of the expected cost (not in the
 * paper; built on pw_qaoa_amp_grad). d_bits (device, packed like pw_sample's
 * output) holds n_samples >= 1 bitstrings drawn from p(x) = |amp(C, x)|^2 of
 * the noiseless QAOA circuit, e.g. by pw_sample on the same circuit. With the
 * diagonal cost C(x) = sum_e w_e z_u z_v + sum_j h_j z_j, z = 1 - 2x (the
 * energy of the cost Hamiltonian), and the score d log p = 2 Re(conj(amp)
 * d amp) / |amp|^2, writes d_out (device, 1 + 2p doubles): the sample mean of
 * C, then N/(N-1) (mean(C score) - mean(C) mean(score)) for gammas[0..p-1]
 * and betas[0..p-1] (the sample-mean baseline, unbiased; the plain mean of
 * C score when N = 1). Reductions run in FP64 in a fixed order, so the result
 * is deterministic. Allocates and frees scratch of about (2p + 1) * 16 bytes
 * per sample, synchronises the stream; errors as pw_qaoa_amp_grad, and
 * PW_ERR_ARG for n_samples == 0. */
int pw_qaoa_cost_grad(int n, int n_edges, const int* edges, const double* w, const double* h, int p,
                      const double* gammas, const double* betas, const pw_plan_opts* opts,
                      uint64_t n_samples, const uint64_t* d_bits, double* d_out, void* stream);

/* Allocation-free variant of pw_sample, for callers that cannot allocate
 * device memory: for example a process whose device memory is entirely
 * reserved by a framework's own memory pool, or code that must not allocate
 * inside its sampling loop. (The paper has no counterpart; this is an
 * interface of this library.) The caller passes the plan and the output buffer
 * d_out_bits (n_samples * ceil(n/64) uint64, device) exactly as for pw_sample;
 * the kernel's scratch (a copy of the plan tables and the two draw counters)
 * lives in one fixed 2 MiB array in device memory that the library holds on
 * every device it is loaded on, until the process exits. Plans whose tables do
 * not fit (pw_plan_stats().device_bytes > 2 MiB - 256 B) are rejected with
 * PW_ERR_TOO_LARGE. No cudaMalloc, cudaFree or allocating library routine is
 * called. The first call on a device looks up the array's device address with
 * that device current. Every
 * call reloads the plan tables and zeroes the counters in the shared array, so
 * calls that overlap on the GPU (on different streams, or from different
 * threads) race and must be serialised by the caller. The results are those of
 * pw_sample for the same arguments. */
int pw_sample_static(const pw_plan* plan, uint64_t seed, uint64_t first_sample, uint64_t n_samples,
                     uint64_t* d_out_bits, void* stream, pw_run_stats_t* stats);

/* ----------------------------------------------------- dense sweep passes */

/* Index bits of a dense pass. Tensor entry i (complex) has index bits
 * b_0 .. b_{W-1}; the pass acts on the k tile bits. */
typedef struct {
    int width_bits;      /* W: each tensor holds 2^W complex entries, tile_bits + 7 <= W <= 31 */
    int tile_bits;       /* k: 5 or 6 */
    int tile_pos[8];     /* operator index bit j is tensor index bit tile_pos[j] */
    int row_pos[7];      /* seven more distinct bits: the 128 rows of one GEMM tile (put
                            the lowest free bits here: consecutive rows, consecutive
                            addresses) */
    int swizzled;        /* 1: entry i is stored at position i ^ ((i >> 4) & 15) */
    int n_diag;          /* diagonal factors applied after the operator, 0..4 */
    int diag_bits[4];    /* bits read by factor d, 0..5 */
    int diag_pos[4][5];  /* factor d's table index bit b is tensor index bit diag_pos[d][b] */
    int reserved[8];
} pw_dense_desc;

/* One dense pass of the sweep contraction (Sec. 2; the per-gate contraction's
 * big steps as GEMMs, not in the paper): for each of n_tensors tensors x
 * (device, 2^W complex FP32 entries each, interleaved (re, im), updated in
 * place) with its operator Op (device d_ops: 2^k x 2^k complex FP32 per
 * tensor, row-major, Op[t'][t]) and its diagonal tables (device d_diag:
 * n_diag x 32 complex FP32 per tensor; nullable when n_diag = 0):
 *   x'[i] = prod_d D_d[bits of i at diag_pos[d]] * sum_t Op[t'(i)][t] x[i with tile bits = t],
 * t'(i) being i's tile bits. gemm picks the arithmetic (PW_GEMM_*): the
 * tensor-core kinds run tcgen05 MMAs with FP32 accumulation in tensor memory,
 * the operator and the tensor entries split into BF16 terms. Allocates and
 * frees an error flag, synchronises the stream.
 * PW_ERR_ARG for invalid bit sets, PW_ERR_TIMEOUT if a bounded wait of the
 * tensor-core kernel ran out. */
int pw_dense_apply(int gemm, const pw_dense_desc* desc, uint64_t n_tensors, float* d_tensors,
                   const float* d_ops, const float* d_diag, void* stream);

/* Measured arithmetic rate of the current device's CUDA cores (not in the
 * paper: the denominator of the roofline fractions of the SIMT contraction
 * kernels). Runs a probe kernel of independent fused multiply-add chains in
 * FP32 (precision = PW_PREC_FP32) or FP64 (PW_PREC_FP64) on every SM for
 * about 30 ms, five times after a calibration, on stream (NULL = legacy), and
 * writes the best rate in TFLOP/s (2 flops per FMA) to *tflops. Synchronises
 * the stream; allocates nothing. */
int pw_device_fma_rate(int precision, void* stream, double* tflops);

/* Device memory of the library's internal buffers (plan tables and
 * counters, staging of pw_sample_host, the HBM engine's frontiers and
 * operators, gradient and autotune scratch): cudaMalloc / cudaFree unless
 * the caller registers an allocator (not in the paper: the boundary's
 * convention that the caller's memory manager, e.g. a framework's caching
 * allocator, owns all device memory). alloc(bytes, device, stream, ctx)
 * returns device memory on `device` (the current device) or NULL (the call
 * then fails with PW_ERR_OOM); free(ptr, device, stream, ctx) releases it;
 * stream is NULL (the legacy stream). Process-wide; both NULL restores
 * cudaMalloc / cudaFree. A buffer is always released by the pair that
 * allocated it, after the device has gone idle. pw_sample_static allocates
 * nothing either way. */
typedef void* (*pw_alloc_fn)(uint64_t bytes, int device, void* stream, void* ctx);
typedef void (*pw_free_fn)(void* ptr, int device, void* stream, void* ctx);
int pw_set_allocator(pw_alloc_fn alloc, pw_free_fn free, void* ctx);

/* Thread-local message describing the last failure of this thread. */
const char* pw_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PW_H */

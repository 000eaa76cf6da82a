// Exact derivatives of amplitudes with respect to circuit parameters.
//
// By the product rule, if each gate A_i depends on at most one parameter
// theta_k(i), then d amp(x) / d theta_k = sum over the gates i of parameter k
// of the amplitude (Sec. 2) of the circuit with A_i replaced by dA_i / d theta_k
// (pw_amp_grad: the caller gives dA_i). A replaced diagonal gate stays
// diagonal and a one-qubit gate stays a one-qubit gate, so each such circuit is
// planned and contracted by the pilot-wave amplitude path like the original.
//
// For the QAOA circuit of App. D (pw_qaoa_amp_grad) every angle enters through
// gates exp(-i t G) with an involutory generator G (Z_u Z_v, Z_j, X_j) and t
// proportional to the angle with coefficient w_e, h_j or 1; the derivative
// matrix is that coefficient times -i G A = exp(-i (t + pi/2) G) (the gate
// advanced by a quarter turn, the parameter-shift rule for amplitudes), formed
// exactly by swapping rows and multiplying by +-i, with the coefficient applied
// to the amplitude in FP64. The QAOA gradient takes p(|E| + n) contractions,
// p(|E| + 2n) with fields h. Gradients are not part of the paper's method.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "pw_internal.h"

using pw::cd;

namespace {

int grad_cuda_fail(cudaError_t e, const char* what) {
    return pw::set_error(PW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// grad[k * ncol + col] += coef * amp[k] for k < n (complex, interleaved).
__global__ void axpy_column(const double2* __restrict__ amp, double coef, double2* __restrict__ grad,
                            int ncol, int col, uint64_t n) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const double2 a = amp[k];
        double2 g = grad[k * ncol + col];
        g.x = fma(coef, a.x, g.x);
        g.y = fma(coef, a.y, g.y);
        grad[k * ncol + col] = g;
    }
}

// -i G A for the gate's generator G on its own local index (bit i = qubit i).
std::vector<cd> quarter_turn(const pw::Op& op, bool x_generator) {
    const int d = op.dim();
    std::vector<cd> out((size_t)d * d);
    const cd mi(0.0, -1.0);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            if (x_generator) {   // -i X A: row r of the result is row r^1 of A
                out[r * d + c] = mi * op.mats[(r ^ 1) * d + c];
            } else {             // -i Z..Z A: sign (-1)^(parity of r)
                const bool odd = __builtin_popcount((unsigned)r) & 1;
                out[r * d + c] = (odd ? -mi : mi) * op.mats[r * d + c];
            }
        }
    return out;
}

struct PlanGuard {
    pw_plan* p = nullptr;
    ~PlanGuard() { pw_plan_destroy(p); }
};

// One concurrent lane of derivative terms: a non-blocking stream with its own
// amplitude scratch and derivative accumulator (lanes are summed in a fixed
// order at the end, so the result does not depend on their scheduling).
struct Lane {
    Lane() = default;
    Lane(const Lane&) = delete;
    Lane& operator=(const Lane&) = delete;
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    double2* amp = nullptr;   // n_strings
    double2* acc = nullptr;   // n_strings * ncol
    ~Lane() {
        if (s) cudaStreamSynchronize(s);
        if (done) cudaEventDestroy(done);
        if (s) cudaStreamDestroy(s);
        pw::dev_free(amp);
        pw::dev_free(acc);
    }
};

// grad[i] = sum over lanes l (in order) of acc_l[i], i < count (complex).
__global__ void sum_lanes(const double2* const* __restrict__ acc, int lanes, double2* __restrict__ grad,
                         uint64_t count) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        double2 g = acc[0][i];
        for (int l = 1; l < lanes; ++l) {
            g.x += acc[l][i].x;
            g.y += acc[l][i].y;
        }
        grad[i] = g;
    }
}

constexpr int kMaxLanes = 16;
constexpr int kRoundPerLane = 16;

struct CircuitGuard {
    pw_circuit* c = nullptr;
    ~CircuitGuard() { pw_circuit_destroy(c); }
};

// One derivative term: the circuit with op `op`'s matrix replaced by `mat`,
// whose amplitude times `coef` adds to derivative column `col`.
struct Term {
    int op, col;
    double coef;
    std::vector<cd> mat;
};

// amp(C, x) of the circuit into d_amp (nullable). Plans it first, so that an
// unsupported structure is reported before any device work.
int base_amplitudes(const pw_circuit* base, const pw_plan_opts* opts, uint64_t n_strings, const uint64_t* d_bits,
                    double* d_amp, cudaStream_t st) {
    PlanGuard pl;
    int rc = pw_plan_build(base, opts, &pl.p);
    if (rc || n_strings == 0) return rc;
    if (d_amp && (rc = pw_amplitudes(pl.p, (int)base->ops.size(), n_strings, d_bits, d_amp, st))) return rc;
    const cudaError_t e = cudaStreamSynchronize(st);   // before the plan's tables are freed
    return e == cudaSuccess ? PW_OK : grad_cuda_fail(e, "cudaStreamSynchronize");
}

// d_grad[k][col] = sum over the terms of that column of coef * amp(term's circuit, x_k),
// for n_strings strings and ncol columns (complex, row-major).
int run_terms(const pw_circuit* base, const std::vector<Term>& terms, int ncol, const pw_plan_opts* opts,
              uint64_t n_strings, const uint64_t* d_bits, double* d_grad, cudaStream_t st) {
    const int n_ops = (int)base->ops.size();
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n_strings + 255) / 256;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)std::max(nsm, 1) * 8);
    cudaError_t e;

    // The terms are spread over lanes: lane l takes terms l, l + L,
    // l + 2L, ... in order, on its own host thread (planning the shifted
    // circuit, uploading its tables, launching its contraction and the
    // accumulation) and its own non-blocking stream with its own amplitude
    // scratch and FP64 accumulator. Contractions of different terms overlap on
    // the device and the host work runs in parallel; the lanes are summed in a
    // fixed order at the end, so the result does not depend on scheduling.
    const int n_terms = (int)terms.size();
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    // each lane holds n_strings * (ncol + 1) complex values: at most 1 GiB for all lanes
    const uint64_t lane_bytes = n_strings * (uint64_t)(ncol + 1) * sizeof(double2);
    const int by_memory = (int)std::max<uint64_t>(1, std::min<uint64_t>(kMaxLanes, (uint64_t(1) << 30) / lane_bytes));
    // plans on the HBM engine hold frontier buffers of up to 16 GB each: their
    // terms run one after another, each plan released after its term
    bool hbm = false;
    {
        pw_plan* probe = nullptr;
        if (pw_plan_build(base, opts, &probe) == PW_OK) {
            hbm = probe->hp.engine == 1;
            pw_plan_destroy(probe);
        }
    }
    const int n_lanes = hbm ? 1 : std::max(1, std::min({kMaxLanes, hw, n_terms, by_memory}));

    cudaEvent_t ready = nullptr;
    if ((e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming)) != cudaSuccess)
        return grad_cuda_fail(e, "cudaEventCreate");
    struct EventGuard {
        cudaEvent_t ev;
        ~EventGuard() { cudaEventDestroy(ev); }
    } ready_guard{ready};
    if ((e = cudaEventRecord(ready, st)) != cudaSuccess) return grad_cuda_fail(e, "cudaEventRecord");
    std::vector<Lane> lanes(n_lanes);
    for (Lane& ln : lanes) {
        if ((e = cudaStreamCreateWithFlags(&ln.s, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming)) != cudaSuccess)
            return grad_cuda_fail(e, "gradient lane set-up");
        if (int rc0 = pw::dev_alloc(reinterpret_cast<void**>(&ln.amp), n_strings * sizeof(double2), "gradient lane"))
            return rc0;
        if (int rc0 = pw::dev_alloc(reinterpret_cast<void**>(&ln.acc), n_strings * ncol * sizeof(double2), "gradient lane"))
            return rc0;
        if ((e = cudaStreamWaitEvent(ln.s, ready, 0)) != cudaSuccess ||
            (e = cudaMemsetAsync(ln.acc, 0, n_strings * ncol * sizeof(double2), ln.s)) != cudaSuccess)
            return grad_cuda_fail(e, "gradient lane set-up");
    }

    // A round's plans stay alive until every lane has finished the round
    // (freeing device memory synchronises the whole device, which would stall
    // the other lanes); a round holds at most kRoundPerLane terms per lane.
    std::vector<pw_plan*> plans(n_terms, nullptr);
    struct PlansGuard {
        std::vector<pw_plan*>& v;
        std::vector<Lane>& lanes;
        void release(int b, int e) {
            for (Lane& ln : lanes)
                if (ln.s) cudaStreamSynchronize(ln.s);
            for (int i = b; i < e; ++i) {
                pw_plan_destroy(v[i]);
                v[i] = nullptr;
            }
        }
        ~PlansGuard() { release(0, (int)v.size()); }
    } plans_guard{plans, lanes};
    std::vector<int> codes(n_lanes, 0);
    std::vector<std::string> msgs(n_lanes);
    auto run_lane = [&](int l, int b, int e_) {
        Lane& ln = lanes[l];
        // the runtime keeps the current device per host thread: a new lane
        // thread starts on device 0, while the plans, streams and scratch
        // of this call belong to the caller's device
        if (const cudaError_t de = cudaSetDevice(dev); de != cudaSuccess) {
            codes[l] = grad_cuda_fail(de, "cudaSetDevice");
            msgs[l] = pw_last_error();
            return;
        }
        pw_circuit shifted;
        shifted.n = base->n;
        for (int i = b + l; i < e_ && !codes[l]; i += n_lanes) {
            const Term& tm = terms[i];
            shifted.ops = base->ops;
            shifted.ops[tm.op].mats = tm.mat;
            int r;
            try {
                r = pw_plan_build(&shifted, opts, &plans[i]);
            } catch (...) {
                r = pw::set_error(PW_ERR_OOM, "allocation failed while planning a derivative term");
            }
            if (!r) r = pw_amplitudes(plans[i], n_ops, n_strings, d_bits, reinterpret_cast<double*>(ln.amp), ln.s);
            if (!r) {
                axpy_column<<<blocks, 256, 0, ln.s>>>(ln.amp, tm.coef, ln.acc, ncol, tm.col, n_strings);
                const cudaError_t le = cudaGetLastError();
                if (le != cudaSuccess) r = grad_cuda_fail(le, "axpy_column launch");
            }
            if (r) {
                codes[l] = r;
                msgs[l] = pw_last_error();
            }
        }
    };
    const int round = hbm ? 1 : n_lanes * kRoundPerLane;
    for (int b = 0; b < n_terms; b += round) {
        const int e_ = std::min(n_terms, b + round);
        std::vector<std::thread> pool;
        for (int l = 1; l < n_lanes; ++l) pool.emplace_back(run_lane, l, b, e_);
        run_lane(0, b, e_);
        for (auto& th : pool) th.join();
        for (int l = 0; l < n_lanes; ++l)
            if (codes[l]) return pw::set_error(codes[l], msgs[l]);
        plans_guard.release(b, e_);
    }

    // d_grad = the lanes' accumulators summed in lane order, on the caller's stream
    std::vector<const double2*> acc_ptrs(n_lanes);
    for (int l = 0; l < n_lanes; ++l) acc_ptrs[l] = lanes[l].acc;
    const double2** d_ptrs = nullptr;
    if (int rc0 = pw::dev_alloc(reinterpret_cast<void**>(&d_ptrs), n_lanes * sizeof(double2*), "lane table")) return rc0;
    struct PtrFree {
        const double2** q;
        ~PtrFree() { pw::dev_free(const_cast<double2**>(q)); }
    } ptr_free{d_ptrs};
    if ((e = cudaMemcpy(d_ptrs, acc_ptrs.data(), n_lanes * sizeof(double2*), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess)
        return grad_cuda_fail(e, "cudaMemcpy");
    for (Lane& ln : lanes) {
        if ((e = cudaEventRecord(ln.done, ln.s)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ln.done, 0)) != cudaSuccess)
            return grad_cuda_fail(e, "gradient lane join");
    }
    const uint64_t total = n_strings * ncol;
    const unsigned sblocks = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)std::max(nsm, 1) * 8);
    sum_lanes<<<sblocks, 256, 0, st>>>(d_ptrs, n_lanes, reinterpret_cast<double2*>(d_grad), total);
    if ((e = cudaGetLastError()) != cudaSuccess) return grad_cuda_fail(e, "sum_lanes launch");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return grad_cuda_fail(e, "cudaStreamSynchronize");
    return PW_OK;
}


}  // namespace

extern "C" int pw_qaoa_amp_grad(int n, int n_edges, const int* edges, const double* w, const double* h, int p,
                                const double* gammas, const double* betas, const pw_plan_opts* opts,
                                uint64_t n_strings, const uint64_t* d_bits, double* d_amp, double* d_grad,
                                void* stream) {
    if (p < 1) return pw::set_error(PW_ERR_ARG, "p must be >= 1");
    if (n_strings && (!d_bits || !d_grad)) return pw::set_error(PW_ERR_ARG, "null argument");
    CircuitGuard base;
    int rc = pw_circuit_qaoa(n, n_edges, edges, w, h, p, gammas, betas, 0.0, 0.0, &base.c);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((rc = base_amplitudes(base.c, opts, n_strings, d_bits, d_amp, st)) || n_strings == 0) return rc;
    // per layer: the edges' RZZ (generator Z_u Z_v, weight w_e), the fields' RZ
    // (Z_j, h_j), the mixers' RX (X_j, 1)
    const int per_layer = n_edges + (h ? n : 0) + n;
    std::vector<Term> terms;
    for (int l = 0; l < p; ++l)
        for (int t = 0; t < per_layer; ++t) {
            const bool mixer = t >= per_layer - n;
            const double coef = mixer ? 1.0 : t < n_edges ? w[t] : h[t - n_edges];
            const int op = n + l * per_layer + t;
            if (coef != 0.0) terms.push_back({op, mixer ? p + l : l, coef, quarter_turn(base.c->ops[op], mixer)});
        }
    return run_terms(base.c, terms, 2 * p, opts, n_strings, d_bits, d_grad, st);
}

extern "C" int pw_amp_grad(const pw_circuit* c, int n_params, const int* param_of_op, const double* dmats,
                           const pw_plan_opts* opts, uint64_t n_strings, const uint64_t* d_bits, double* d_amp,
                           double* d_grad, void* stream) {
    if (!c || !param_of_op) return pw::set_error(PW_ERR_ARG, "null argument");
    if (n_params < 1) return pw::set_error(PW_ERR_ARG, "n_params must be >= 1");
    if (n_strings && (!d_bits || !d_grad)) return pw::set_error(PW_ERR_ARG, "null argument");
    std::vector<Term> terms;
    size_t at = 0;
    for (int i = 0; i < (int)c->ops.size(); ++i) {
        const int k = param_of_op[i];
        if (k < -1 || k >= n_params) return pw::set_error(PW_ERR_ARG, "param_of_op entry out of range");
        if (k < 0) continue;
        const pw::Op& op = c->ops[i];
        if (op.kind != pw::OP_GATE) return pw::set_error(PW_ERR_ARG, "a parameterised operation must be a gate");
        if (!dmats) return pw::set_error(PW_ERR_ARG, "null argument");
        const int d = op.dim();
        Term tm{i, k, 1.0, std::vector<cd>((size_t)d * d)};
        for (int j = 0; j < d * d; ++j, ++at) {
            tm.mat[j] = cd(dmats[2 * at], dmats[2 * at + 1]);
            if (!std::isfinite(tm.mat[j].real()) || !std::isfinite(tm.mat[j].imag()))
                return pw::set_error(PW_ERR_NUMERIC, "non-finite derivative entry");
        }
        terms.push_back(std::move(tm));
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = base_amplitudes(c, opts, n_strings, d_bits, d_amp, st);
    if (rc || n_strings == 0) return rc;
    return run_terms(c, terms, n_params, opts, n_strings, d_bits, d_grad, st);
}

// ------------------------------------------- score-function cost gradient
// For samples x_1..x_N drawn from p(x) = |amp(x)|^2 and the diagonal cost
// C(x) = <x|H_C|x> = sum_e w_e z_u z_v + sum_j h_j z_j (z = 1 - 2 x), the
// gradient of E[C] is E[C(x) d log p(x)] with d log p = 2 Re(conj(amp) d amp) /
// |amp|^2 (the score). With the sample-mean baseline the unbiased estimate is
//   N/(N-1) * (mean(C * score) - mean(C) * mean(score)).
namespace {

constexpr int kCostThreads = 256;

// One thread per sample; a block's sums of C, score_j and C * score_j go to
// partial[block][1 + 4p] (fixed-order tree reductions: the result does not
// depend on scheduling).
__global__ void cost_score_partials(const uint64_t* __restrict__ bits, int words, const double2* __restrict__ amp,
                                   const double2* __restrict__ grad, int ncol, const int* __restrict__ edges,
                                   const double* __restrict__ w, int n_edges, const double* __restrict__ h, int n,
                                   uint64_t count, double* __restrict__ partial) {
    extern __shared__ double red[];   // [1 + 2 ncol][kCostThreads]
    const int nv = 1 + 2 * ncol;
    const uint64_t k = blockIdx.x * (uint64_t)kCostThreads + threadIdx.x;
    double c = 0.0;
    double inv_p = 0.0;
    double2 a = make_double2(0.0, 0.0);
    if (k < count) {
        const uint64_t* x = bits + k * words;
        auto z = [&](int q) { return ((x[q >> 6] >> (q & 63)) & 1ull) ? -1.0 : 1.0; };
        for (int e = 0; e < n_edges; ++e) c = fma(w[e], z(edges[2 * e]) * z(edges[2 * e + 1]), c);
        if (h)
            for (int j = 0; j < n; ++j) c = fma(h[j], z(j), c);
        a = amp[k];
        const double pr = a.x * a.x + a.y * a.y;
        inv_p = pr > 0.0 ? 1.0 / pr : 0.0;   // a string of zero probability is never drawn
    }
    red[threadIdx.x] = k < count ? c : 0.0;
    for (int j = 0; j < ncol; ++j) {
        double s = 0.0;
        if (k < count) {
            const double2 g = grad[k * ncol + j];
            s = 2.0 * (a.x * g.x + a.y * g.y) * inv_p;
        }
        red[(1 + j) * kCostThreads + threadIdx.x] = s;
        red[(1 + ncol + j) * kCostThreads + threadIdx.x] = k < count ? c * s : 0.0;
    }
    __syncthreads();
    for (int half = kCostThreads / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half)
            for (int v = 0; v < nv; ++v) red[v * kCostThreads + threadIdx.x] += red[v * kCostThreads + threadIdx.x + half];
        __syncthreads();
    }
    if (threadIdx.x < nv) partial[blockIdx.x * (uint64_t)nv + threadIdx.x] = red[threadIdx.x * kCostThreads];
}

// out[0] = mean C; out[1 + j] = the baselined score-function estimate.
__global__ void cost_score_finish(const double* __restrict__ partial, unsigned blocks, int ncol, uint64_t count,
                                  double* __restrict__ out) {
    const int nv = 1 + 2 * ncol;
    const double inv_n = 1.0 / (double)count;
    double sum_c = 0.0;
    for (unsigned b = 0; b < blocks; ++b) sum_c += partial[b * (uint64_t)nv];
    for (int j = threadIdx.x; j < ncol; j += blockDim.x) {
        double s = 0.0, cs = 0.0;
        for (unsigned b = 0; b < blocks; ++b) {
            s += partial[b * (uint64_t)nv + 1 + j];
            cs += partial[b * (uint64_t)nv + 1 + ncol + j];
        }
        const double mc = sum_c * inv_n;
        out[1 + j] = count > 1 ? ((double)count / (double)(count - 1)) * (cs * inv_n - mc * (s * inv_n)) : cs;
    }
    if (threadIdx.x == 0) out[0] = sum_c * inv_n;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { pw::dev_free(p); }
};

}  // namespace

extern "C" int pw_qaoa_cost_grad(int n, int n_edges, const int* edges, const double* w, const double* h, int p,
                                 const double* gammas, const double* betas, const pw_plan_opts* opts,
                                 uint64_t n_samples, const uint64_t* d_bits, double* d_out, void* stream) {
    if (p < 1) return pw::set_error(PW_ERR_ARG, "p must be >= 1");
    if (n_samples == 0) return pw::set_error(PW_ERR_ARG, "n_samples must be >= 1");
    if (!d_bits || !d_out || (n_edges > 0 && (!edges || !w))) return pw::set_error(PW_ERR_ARG, "null argument");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ncol = 2 * p;
    const unsigned blocks = (unsigned)((n_samples + kCostThreads - 1) / kCostThreads);
    const size_t nv = 1 + 2 * (size_t)ncol;
    const size_t smem = nv * kCostThreads * sizeof(double);
    if (smem > 227 * 1024) return pw::set_error(PW_ERR_TOO_LARGE, "too many angles for one reduction block");
    const size_t amp_b = n_samples * sizeof(double2), grad_b = n_samples * ncol * sizeof(double2);
    const size_t part_b = (size_t)blocks * nv * sizeof(double);
    const size_t edge_b = (size_t)n_edges * 2 * sizeof(int), w_b = (size_t)n_edges * sizeof(double);
    const size_t h_b = h ? (size_t)n * sizeof(double) : 0;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    DevBuf buf;
    if (int rc0 = pw::dev_alloc(&buf.p, up(amp_b) + up(grad_b) + up(part_b) + up(edge_b) + up(w_b) + up(h_b),
                                "cost gradient scratch"))
        return rc0;
    cudaError_t e = cudaSuccess;
    struct SyncOnExit {   // destroyed before the scratch: nothing is freed under running copies or kernels
        cudaStream_t s;
        ~SyncOnExit() { cudaStreamSynchronize(s); }
    } sync_on_exit{st};
    char* base = static_cast<char*>(buf.p);
    double2* d_amp = reinterpret_cast<double2*>(base);
    double2* d_grad = reinterpret_cast<double2*>(base + up(amp_b));
    double* d_part = reinterpret_cast<double*>(base + up(amp_b) + up(grad_b));
    int* d_edges = reinterpret_cast<int*>(base + up(amp_b) + up(grad_b) + up(part_b));
    double* d_w = reinterpret_cast<double*>(base + up(amp_b) + up(grad_b) + up(part_b) + up(edge_b));
    double* d_h = h ? reinterpret_cast<double*>(base + up(amp_b) + up(grad_b) + up(part_b) + up(edge_b) + up(w_b))
                    : nullptr;
    if (n_edges > 0) {
        if ((e = cudaMemcpyAsync(d_edges, edges, edge_b, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_w, w, w_b, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return grad_cuda_fail(e, "cudaMemcpyAsync(graph)");
    }
    if (h && (e = cudaMemcpyAsync(d_h, h, h_b, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return grad_cuda_fail(e, "cudaMemcpyAsync(fields)");
    int rc = pw_qaoa_amp_grad(n, n_edges, edges, w, h, p, gammas, betas, opts, n_samples, d_bits,
                              reinterpret_cast<double*>(d_amp), reinterpret_cast<double*>(d_grad), stream);
    if (rc) return rc;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(cost_score_partials, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
        return grad_cuda_fail(e, "cudaFuncSetAttribute");
    cost_score_partials<<<blocks, kCostThreads, smem, st>>>(d_bits, (n + 63) / 64, d_amp, d_grad, ncol, d_edges, d_w,
                                                            n_edges, d_h, n, n_samples, d_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return grad_cuda_fail(e, "cost_score_partials launch");
    cost_score_finish<<<1, 64, 0, st>>>(d_part, blocks, ncol, n_samples, d_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return grad_cuda_fail(e, "cost_score_finish launch");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return grad_cuda_fail(e, "cudaStreamSynchronize");
    return PW_OK;
}

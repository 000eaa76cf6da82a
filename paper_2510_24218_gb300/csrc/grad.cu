// Exact derivatives of QAOA amplitudes with respect to the angles, by the
// parameter-shift rule for amplitudes.
//
// Every angle enters the QAOA circuit of App. D through gates exp(-i t G) with
// an involutory generator G (G^2 = I: Z_u Z_v, Z_j, X_j). For such a gate
// d/dt exp(-i t G) = -i G exp(-i t G) = exp(-i (t + pi/2) G), so
//
//   d amp(x) / d gamma_l = sum_e w_e amp_{e,l}(x) + sum_j h_j amp_{j,l}(x),
//   d amp(x) / d beta_l  = sum_j amp'_{j,l}(x),
//
// where each amp_* is the amplitude (Sec. 2) of the same circuit with the one
// gate replaced by -i G times itself (its angle advanced by pi/2). Those
// circuits have the structure of the original, so each is planned and
// contracted by the pilot-wave amplitude path; the replaced matrix is the
// original one with rows swapped and entries multiplied by +-i, exact in
// floating point. This is not the paper's method (it gives no gradients); it
// reuses the amplitude contraction 2p(|E| + 2n) times (n without fields).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
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
void advance_quarter_turn(pw::Op& op, bool x_generator) {
    const int d = op.dim();
    std::vector<cd> A(op.mats.begin(), op.mats.begin() + d * d);
    const cd mi(0.0, -1.0);
    for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
            if (x_generator) {   // -i X A: row r of the result is row r^1 of A
                op.mats[r * d + c] = mi * A[(r ^ 1) * d + c];
            } else {             // -i Z..Z A: sign (-1)^(parity of r)
                const bool odd = __builtin_popcount((unsigned)r) & 1;
                op.mats[r * d + c] = (odd ? -mi : mi) * A[r * d + c];
            }
        }
}

struct PlanGuard {
    pw_plan* p = nullptr;
    ~PlanGuard() { pw_plan_destroy(p); }
};

struct Scratch {
    double2* amp = nullptr;
    cudaEvent_t done = nullptr;
    ~Scratch() {
        if (done) cudaEventDestroy(done);
        cudaFree(amp);
    }
};

struct CircuitGuard {
    pw_circuit* c = nullptr;
    ~CircuitGuard() { pw_circuit_destroy(c); }
};

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
    const int n_ops = (int)base.c->ops.size();
    const int per_layer = n_edges + (h ? n : 0) + n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ncol = 2 * p;

    // the unshifted amplitudes (plans the circuit first: an unsupported
    // structure is reported before any device work)
    {
        PlanGuard pl;
        if ((rc = pw_plan_build(base.c, opts, &pl.p))) return rc;
        if (n_strings == 0) return PW_OK;
        if (d_amp && (rc = pw_amplitudes(pl.p, n_ops, n_strings, d_bits, d_amp, stream))) return rc;
        cudaError_t e = cudaStreamSynchronize(st);   // before the plan's tables are freed
        if (e != cudaSuccess) return grad_cuda_fail(e, "cudaStreamSynchronize");
    }
    cudaError_t e = cudaMemsetAsync(d_grad, 0, n_strings * ncol * 2 * sizeof(double), st);
    if (e != cudaSuccess) return grad_cuda_fail(e, "cudaMemsetAsync(grad)");
    Scratch sc;
    if ((e = cudaMalloc(&sc.amp, n_strings * sizeof(double2))) != cudaSuccess)
        return grad_cuda_fail(e, "cudaMalloc(grad scratch)");
    if ((e = cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming)) != cudaSuccess)
        return grad_cuda_fail(e, "cudaEventCreate");

    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n_strings + 255) / 256;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)std::max(nsm, 1) * 8);

    // Depth-2 pipeline: the next shifted circuit is planned on the host while
    // the previous one's contraction runs; a plan is destroyed only after the
    // event recorded behind its work has completed.
    pw_circuit shifted;
    shifted.n = base.c->n;
    PlanGuard prev;
    struct SyncOnExit {   // destroyed first: no plan or scratch is freed under running work
        cudaStream_t s;
        ~SyncOnExit() { cudaStreamSynchronize(s); }
    } sync_on_exit{st};
    for (int l = 0; l < p; ++l) {
        const int first = n + l * per_layer;
        for (int t = 0; t < per_layer; ++t) {
            const bool mixer = t >= per_layer - n;
            const double coef = mixer ? 1.0 : t < n_edges ? w[t] : h[t - n_edges];
            if (coef == 0.0) continue;
            shifted.ops = base.c->ops;
            advance_quarter_turn(shifted.ops[first + t], mixer);
            PlanGuard cur;
            if ((rc = pw_plan_build(&shifted, opts, &cur.p))) return rc;
            if (prev.p && (e = cudaEventSynchronize(sc.done)) != cudaSuccess)
                return grad_cuda_fail(e, "cudaEventSynchronize");
            if ((rc = pw_amplitudes(cur.p, n_ops, n_strings, d_bits, reinterpret_cast<double*>(sc.amp), stream)))
                return rc;
            axpy_column<<<blocks, 256, 0, st>>>(sc.amp, coef, reinterpret_cast<double2*>(d_grad), ncol,
                                                mixer ? p + l : l, n_strings);
            if ((e = cudaGetLastError()) != cudaSuccess) return grad_cuda_fail(e, "axpy_column launch");
            if ((e = cudaEventRecord(sc.done, st)) != cudaSuccess) return grad_cuda_fail(e, "cudaEventRecord");
            std::swap(prev.p, cur.p);   // cur now holds the plan whose work has finished
        }
    }
    // the scratch and the last plan are freed on return: wait for their work
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return grad_cuda_fail(e, "cudaStreamSynchronize");
    return PW_OK;
}

// Measured throughput of the device's FP32 and FP64 fused multiply-add pipes
// (CUDA cores, not tensor cores). The SIMT contraction kernels of this
// library are bound by these pipes, so their roofline fractions are taken
// against the measured rate rather than a figure derived from unit counts and
// the nominal clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "pw_internal.h"

namespace pw {
namespace {

// Every thread runs 8 independent FMA chains x <- x * a + b (a just below 1,
// b small: the values stay bounded and no chain can be simplified away).
template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(R* sink, int iters, R a, R b) {
    R x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (R)(threadIdx.x & 7) + (R)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    R s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == (R)-1) sink[0] = s;   // never true; keeps the chains alive
}

int probe_fail(cudaError_t e, const char* what) {
    return set_error(PW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename R> int run_probe(cudaStream_t st, double* tflops) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return probe_fail(e, "device query");
    const int threads = 256, blocks = std::max(1, nsm) * 8;   // 2048 threads per SM
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return probe_fail(e, "cudaEventCreate");
    }
    const R a = (R)0.999999, b = (R)1e-7;
    auto timed = [&](int iters, float* ms) -> cudaError_t {
        cudaError_t r = cudaEventRecord(e0, st);
        if (r != cudaSuccess) return r;
        fma_probe_kernel<R><<<blocks, threads, 0, st>>>(nullptr, iters, a, b);
        if ((r = cudaGetLastError()) != cudaSuccess) return r;
        if ((r = cudaEventRecord(e1, st)) != cudaSuccess) return r;
        if ((r = cudaEventSynchronize(e1)) != cudaSuccess) return r;
        return cudaEventElapsedTime(ms, e0, e1);
    };
    // calibrate to about 30 ms per timed launch, then the best of five
    int iters = 256;
    float ms = 0.0f;
    for (int rep = 0; rep < 12 && e == cudaSuccess; ++rep) {
        e = timed(iters, &ms);
        if (e != cudaSuccess || ms > 10.0f || iters >= (1 << 26)) break;
        iters *= 4;
    }
    if (e == cudaSuccess && ms > 0.0f) iters = std::max(1, (int)std::min<double>(1e9, iters * (30.0 / ms)));
    float best = 0.0f;
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        float t = 0.0f;
        e = timed(iters, &t);
        if (e == cudaSuccess && (best == 0.0f || t < best)) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return probe_fail(e, "FMA probe");
    if (best <= 0.0f) return set_error(PW_ERR_CUDA, "FMA probe: no time measured");
    const double flops = 2.0 * 32.0 * (double)iters * threads * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    return PW_OK;
}

}  // namespace
}  // namespace pw

extern "C" int pw_device_fma_rate(int precision, void* stream, double* tflops) {
    using namespace pw;
    if (!tflops) return set_error(PW_ERR_ARG, "null argument");
    *tflops = 0.0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (precision == PW_PREC_FP64) return run_probe<double>(st, tflops);
    if (precision == PW_PREC_FP32) return run_probe<float>(st, tflops);
    return set_error(PW_ERR_ARG, "unknown precision");
}

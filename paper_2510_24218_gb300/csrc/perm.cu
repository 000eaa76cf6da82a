// Output permutation of plans whose SWAP-class gates were planned as wire
// relabellings: the kernel writes the chain's bits per wire; output bit q is
// the bit of wire out_wire[q].
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "pw_internal.h"

namespace {

constexpr int kMaxWords = 64;   // 4096 qubits

// One thread per sample: its row is read into registers / local memory and
// rewritten in place.
__global__ void permute_rows(uint64_t* __restrict__ bits, const int* __restrict__ wire, int n, int words,
                             uint64_t count) {
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < count; k += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t* row = bits + k * words;
        uint64_t in[kMaxWords];
        for (int i = 0; i < words; ++i) in[i] = row[i];
        for (int i = 0; i < words; ++i) {
            uint64_t w = 0;
            const int q1 = min(n, (i + 1) * 64);
            for (int q = i * 64; q < q1; ++q) {
                const int s = wire[q];
                w |= ((in[s >> 6] >> (s & 63)) & 1ull) << (q & 63);
            }
            row[i] = w;
        }
    }
}

int perm_fail(cudaError_t e, const char* what) {
    return pw::set_error(PW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

namespace pw {

int permute_output(pw_plan* plan, uint64_t* d_bits, uint64_t n_samples, void* stream) {
    const int n = (int)plan->out_wire.size();
    if (n == 0 || n_samples == 0) return PW_OK;
    const int words = (n + 63) / 64;
    if (words > kMaxWords) return set_error(PW_ERR_TOO_LARGE, "more than 4096 qubits");
    cudaError_t e;
    if (!plan->d_out_wire) {
        int* d = nullptr;
        if ((e = cudaMalloc(&d, sizeof(int) * n)) != cudaSuccess) return perm_fail(e, "cudaMalloc(wire map)");
        // (pageable source: wait for the copy itself, not only for its staging)
        if ((e = cudaMemcpy(d, plan->out_wire.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess) {
            cudaFree(d);
            return perm_fail(e, "cudaMemcpy(wire map)");
        }
        plan->d_out_wire = d;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n_samples + 127) / 128;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)(nsm > 0 ? nsm : 1) * 16);
    permute_rows<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(d_bits, plan->d_out_wire, n, words,
                                                                          n_samples);
    if ((e = cudaGetLastError()) != cudaSuccess) return perm_fail(e, "permute_rows launch");
    return PW_OK;
}

}  // namespace pw

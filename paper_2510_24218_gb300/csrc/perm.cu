// Output permutation of plans whose SWAP-class gates were planned as wire
// relabellings: the kernel writes the chain's bits per wire; output bit q is
// the bit of wire out_wire[q].
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

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

// A device copy of a host map (waits for the copy itself: pageable source).
int upload_map(const std::vector<int>& map, int** out) {
    int* d = nullptr;
    cudaError_t e;
    if (int rc = pw::dev_alloc(reinterpret_cast<void**>(&d), sizeof(int) * map.size(), "wire map")) return rc;
    if ((e = cudaMemcpy(d, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess) {
        pw::dev_free(d);
        return perm_fail(e, "cudaMemcpy(wire map)");
    }
    *out = d;
    return PW_OK;
}

int launch_permute(uint64_t* d_bits, const int* d_map, int n, uint64_t count, cudaStream_t st) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (count + 127) / 128;
    const unsigned blocks = (unsigned)std::min<uint64_t>(want, (uint64_t)(nsm > 0 ? nsm : 1) * 16);
    permute_rows<<<blocks, 128, 0, st>>>(d_bits, d_map, n, (n + 63) / 64, count);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PW_OK : perm_fail(e, "permute_rows launch");
}

}  // namespace

namespace pw {

int permute_output(pw_plan* plan, uint64_t* d_bits, uint64_t n_samples, void* stream) {
    const int n = (int)plan->out_wire.size();
    if (n == 0 || n_samples == 0) return PW_OK;
    if ((n + 63) / 64 > kMaxWords) return set_error(PW_ERR_TOO_LARGE, "more than 4096 qubits");
    int rc;
    if (!plan->d_out_wire && (rc = upload_map(plan->out_wire, &plan->d_out_wire))) return rc;
    return launch_permute(d_bits, plan->d_out_wire, n, n_samples, static_cast<cudaStream_t>(stream));
}

int permute_input(pw_plan* plan, const uint64_t* d_src, uint64_t* d_dst, uint64_t n_strings, void* stream) {
    const int n = (int)plan->out_wire.size();
    if (n == 0 || n_strings == 0) return PW_OK;
    if ((n + 63) / 64 > kMaxWords) return set_error(PW_ERR_TOO_LARGE, "more than 4096 qubits");
    int rc;
    if (!plan->d_in_wire) {
        std::vector<int> inv(n);
        for (int q = 0; q < n; ++q) inv[plan->out_wire[q]] = q;   // wire out_wire[q] holds qubit q
        if ((rc = upload_map(inv, &plan->d_in_wire))) return rc;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaError_t e = cudaMemcpyAsync(d_dst, d_src, n_strings * ((n + 63) / 64) * sizeof(uint64_t),
                                          cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return perm_fail(e, "cudaMemcpyAsync(rows)");
    return launch_permute(d_dst, plan->d_in_wire, n, n_strings, st);
}

}  // namespace pw

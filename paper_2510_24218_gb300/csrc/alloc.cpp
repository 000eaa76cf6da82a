// Device memory of the library's internal buffers. By default cudaMalloc /
// cudaFree; a caller that owns the device memory (a framework's caching
// allocator) registers its own pair with pw_set_allocator. Every buffer is
// released by the pair that allocated it (the pair is recorded per pointer),
// so the allocator may be changed while plans are alive.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <unordered_map>

#include "pw_internal.h"

namespace pw {
namespace {

struct Allocator {
    pw_alloc_fn alloc = nullptr;
    pw_free_fn free = nullptr;
    void* ctx = nullptr;
};

struct Owner {
    pw_free_fn free;
    void* ctx;
    int device;
};

std::mutex g_mu;
Allocator g_alloc;
std::unordered_map<void*, Owner>& owners() {
    static std::unordered_map<void*, Owner> m;
    return m;
}

}  // namespace

int dev_alloc(void** out, size_t bytes, const char* what) {
    *out = nullptr;
    Allocator a;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        a = g_alloc;
    }
    if (!a.alloc) {
        const cudaError_t e = cudaMalloc(out, bytes);
        if (e != cudaSuccess)
            return set_error(e == cudaErrorMemoryAllocation ? PW_ERR_OOM : PW_ERR_CUDA,
                             std::string("cudaMalloc(") + what + "): " + cudaGetErrorString(e));
        return PW_OK;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    void* p = a.alloc(bytes, dev, nullptr, a.ctx);
    if (!p) return set_error(PW_ERR_OOM, std::string("the registered allocator returned no memory for ") + what);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        owners()[p] = Owner{a.free, a.ctx, dev};
    }
    *out = p;
    return PW_OK;
}

void dev_free(void* p) {
    if (!p) return;
    Owner o{};
    bool custom = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = owners().find(p);
        if (it != owners().end()) {
            o = it->second;
            owners().erase(it);
            custom = true;
        }
    }
    if (!custom) {
        cudaFree(p);
        return;
    }
    // the buffer may still be read by work in flight on any stream: the
    // device is idle before it goes back to the caller's allocator
    cudaDeviceSynchronize();
    if (o.free) o.free(p, o.device, nullptr, o.ctx);
}

}  // namespace pw

extern "C" int pw_set_allocator(pw_alloc_fn alloc, pw_free_fn free, void* ctx) {
    using namespace pw;
    if ((alloc == nullptr) != (free == nullptr)) return set_error(PW_ERR_ARG, "alloc and free are set together");
    std::lock_guard<std::mutex> lk(g_mu);
    g_alloc = Allocator{alloc, free, ctx};
    return PW_OK;
}

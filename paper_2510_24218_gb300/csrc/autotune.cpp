// Plan-shape search (pw_autotune): times the sampler over the plan options
// that change only the schedule (engine, readout block size, sweep order,
// threads per chain, chains per launch), one dimension at a time, and keeps
// the fastest; results persist in a JSON-lines cache keyed by the circuit,
// the fixed options and the device.
#include <cuda_runtime.h>

#include <cinttypes>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <string>
#include <vector>

#include "pw_internal.h"

using namespace pw;

namespace {

// FNV-1a over the bytes of the circuit and the options as given (the
// precision, the arithmetic and the fields the caller pinned).
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void bytes(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
    template <typename T> void val(const T& v) { bytes(&v, sizeof(v)); }
};

uint64_t circuit_key(const pw_circuit* c, const pw_plan_opts& o) {
    Fnv f;
    f.val(c->n);
    for (const Op& op : c->ops) {
        f.val(op.kind);
        f.val(op.k);
        for (int q : op.qubits) f.val(q);
        f.bytes(op.mats.data(), op.mats.size() * sizeof(cd));
    }
    for (int v : {o.precision, o.order, o.max_block, o.threads_per_chain, o.chains_per_launch, o.ctas_per_chain,
                  o.engine, o.gemm})
        f.val(v);
    return f.h;
}

std::string device_id(int dev) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "";
    char buf[320];
    std::snprintf(buf, sizeof(buf), "%s sm_%d%d x%d", p.name, p.major, p.minor, p.multiProcessorCount);
    for (char* s = buf; *s; ++s)
        if (*s == '"' || *s == '\\') *s = '_';
    return buf;
}

bool find_num(const std::string& line, const char* name, double* v) {
    const std::string pat = std::string("\"") + name + "\":";
    const size_t at = line.find(pat);
    if (at == std::string::npos) return false;
    const char* s = line.c_str() + at + pat.size();
    char* end = nullptr;
    *v = std::strtod(s, &end);
    return end != s;
}

std::string line_of(const char* key, const std::string& dev, const pw_plan_opts& o, double rate) {
    char buf[768];
    std::snprintf(buf, sizeof(buf),
                  "{\"key\": \"%s\", \"device\": \"%s\", \"engine\": %d, \"max_block\": %d, \"order\": %d, "
                  "\"threads_per_chain\": %d, \"chains_per_launch\": %d, \"samples_per_s\": %.6g}",
                  key, dev.c_str(), o.engine, o.max_block, o.order, o.threads_per_chain, o.chains_per_launch, rate);
    return buf;
}

// The cached options of (key, device), if the cache holds them.
bool cache_lookup(const char* path, const char* key, const std::string& dev, pw_plan_opts* o, double* rate) {
    std::ifstream in(path);
    if (!in) return false;
    const std::string kpat = std::string("\"key\": \"") + key + "\"";
    const std::string dpat = std::string("\"device\": \"") + dev + "\"";
    std::string line;
    bool found = false;
    while (std::getline(in, line)) {
        if (line.find(kpat) == std::string::npos || line.find(dpat) == std::string::npos) continue;
        double e, mb, ord, tpc, cpl, r;
        if (!find_num(line, "engine", &e) || !find_num(line, "max_block", &mb) || !find_num(line, "order", &ord) ||
            !find_num(line, "threads_per_chain", &tpc) || !find_num(line, "chains_per_launch", &cpl) ||
            !find_num(line, "samples_per_s", &r))
            continue;
        o->engine = (int)e;
        o->max_block = (int)mb;
        o->order = (int)ord;
        o->threads_per_chain = (int)tpc;
        o->chains_per_launch = (int)cpl;
        *rate = r;
        found = true;   // (the last matching line wins)
    }
    return found;
}

// Samples per second of a plan built with o: one warm-up call, then the
// fastest of two timed ones; 0 when the options do not plan or run.
double time_opts(const pw_circuit* c, const pw_plan_opts& o, uint64_t n, uint64_t* d_out, cudaStream_t st,
                 cudaEvent_t e0, cudaEvent_t e1) {
    pw_plan* plan = nullptr;
    if (pw_plan_build(c, &o, &plan) != PW_OK) return 0.0;
    double best = 0.0;
    int rc = pw_sample(plan, 0x5eed, 0, n, d_out, nullptr, st, nullptr);
    for (int rep = 0; rep < 2 && rc == PW_OK; ++rep) {
        cudaEventRecord(e0, st);
        rc = pw_sample(plan, 0x5eed, (rep + 1) * n, n, d_out, nullptr, st, nullptr);
        cudaEventRecord(e1, st);
        float ms = 0.0f;
        if (rc == PW_OK && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms > 0.0f) {
            const double r = (double)n / (ms * 1e-3);
            if (r > best) best = r;
        } else {
            best = 0.0;
            break;
        }
    }
    cudaStreamSynchronize(st);
    cudaGetLastError();   // (a shape that does not launch is skipped)
    pw_plan_destroy(plan);
    return best;
}

}  // namespace

extern "C" int pw_autotune(const pw_circuit* c, const pw_plan_opts* base, uint64_t trial_samples, const char* cache_path,
                           void* stream, pw_plan_opts* best, double* samples_per_s, int* from_cache) {
    if (!c || !best) return set_error(PW_ERR_ARG, "null argument");
    pw_plan_opts o{};
    if (base) o = *base;
    if (from_cache) *from_cache = 0;
    if (samples_per_s) *samples_per_s = 0.0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(PW_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    const std::string did = device_id(dev);
    char key[17];
    std::snprintf(key, sizeof(key), "%016" PRIx64, circuit_key(c, o));
    double rate = 0.0;
    if (cache_path && cache_lookup(cache_path, key, did, &o, &rate)) {
        *best = o;
        if (samples_per_s) *samples_per_s = rate;
        if (from_cache) *from_cache = 1;
        return PW_OK;
    }
    // the plan as given sets the output size
    pw_plan* probe = nullptr;
    int rc = pw_plan_build(c, &o, &probe);
    if (rc) return rc;
    pw_plan_stats_t st0;
    pw_plan_stats(probe, &st0);
    pw_plan_destroy(probe);
    const int words = (st0.n_qubits + 63) / 64;
    const uint64_t n = trial_samples ? trial_samples : 16384;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint64_t* d_out = nullptr;
    if (int rc0 = dev_alloc(reinterpret_cast<void**>(&d_out), n * words * sizeof(uint64_t), "autotune output"))
        return rc0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        dev_free(d_out);
        return set_error(PW_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
    rate = time_opts(c, o, n, d_out, st, e0, e1);
    // one dimension at a time, each from the best shape so far; fields the
    // caller set (nonzero) stay as given
    const bool fp32 = o.precision == PW_PREC_FP32;
    auto sweep = [&](int pw_plan_opts::*field, std::initializer_list<int> values) {
        if (base && (base->*field) != 0) return;
        for (int v : values) {
            pw_plan_opts t = o;
            t.*field = v;
            if (v == o.*field) continue;
            const double r = time_opts(c, t, n, d_out, st, e0, e1);
            if (r > rate) {
                rate = r;
                o = t;
            }
        }
    };
    if (fp32) sweep(&pw_plan_opts::engine, {PW_ENGINE_ONCHIP, PW_ENGINE_HBM});
    sweep(&pw_plan_opts::max_block, {4, 6, 8, 12});
    sweep(&pw_plan_opts::order, {PW_ORDER_AUTO, PW_ORDER_NATURAL});
    sweep(&pw_plan_opts::threads_per_chain, {32, 64, 128, 256});
    sweep(&pw_plan_opts::chains_per_launch, {1024, 4096, 8192});
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(d_out);
    if (rate <= 0.0) return set_error(PW_ERR_CUDA, "autotune: no configuration ran");
    *best = o;
    if (samples_per_s) *samples_per_s = rate;
    if (cache_path) {
        std::ofstream out(cache_path, std::ios::app);
        if (!out || !(out << line_of(key, did, o, rate) << '\n'))
            return set_error(PW_ERR_ARG, std::string("autotune: cannot append to ") + cache_path);
    }
    return PW_OK;
}

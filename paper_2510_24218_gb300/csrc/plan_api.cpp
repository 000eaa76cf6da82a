// C ABI of plan construction and inspection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>

#include "pw_internal.h"

using namespace pw;

namespace {

int choose_threads(const HostPlan& hp, int requested) {
    if (requested > 0) {
        if (requested % 32 || requested > 512 || (requested & (requested - 1)))
            return -1;
        return requested;
    }
    long N = 1L << hp.W;
    long t = N / 16;
    t = std::max(32L, std::min(512L, t));
    long pw2 = 32;
    while (pw2 < t) pw2 <<= 1;
    return (int)pw2;
}

}  // namespace

extern "C" {

int pw_plan_build(const pw_circuit* c, const pw_plan_opts* opts, pw_plan** out) {
    if (!c || !out) return set_error(PW_ERR_ARG, "null argument");
    *out = nullptr;
    pw_plan_opts o{};
    if (opts) o = *opts;
    pw_plan* plan = new (std::nothrow) pw_plan();
    if (!plan) return set_error(PW_ERR_OOM, "allocation failed");
    int rc;
    try {
        rc = build_plan(c, o, plan->hp);
    } catch (const std::bad_alloc&) {
        rc = set_error(PW_ERR_OOM, "allocation failed while planning");
    }
    if (rc) {
        delete plan;
        return rc;
    }
    int tpc = choose_threads(plan->hp, o.threads_per_chain);
    if (tpc < 0) {
        delete plan;
        return set_error(PW_ERR_ARG, "threads_per_chain must be a power of two in 32..512");
    }
    plan->hp.threads_per_chain = tpc;
    if (o.chains_per_launch < 0) {
        delete plan;
        return set_error(PW_ERR_ARG, "chains_per_launch must be >= 0");
    }
    plan->hp.chains_per_launch = o.chains_per_launch;
    *out = plan;
    return PW_OK;
}

int pw_plan_stats(const pw_plan* plan, pw_plan_stats_t* s) {
    if (!plan || !s) return set_error(PW_ERR_ARG, "null argument");
    std::memset(s, 0, sizeof(*s));
    const HostPlan& hp = plan->hp;
    s->n_qubits = hp.hdr.n;
    s->n_ops = hp.hdr.n_ops;
    s->n_layers = hp.hdr.P;
    s->n_slots = hp.hdr.S;
    s->width_bits = hp.W;
    s->width_low_bits = hp.W_low;
    s->n_blocks = hp.hdr.K;
    s->sampled_gates = hp.hdr.n_sampled;
    s->threads_per_chain = hp.threads_per_chain;
    s->noisy = hp.noisy ? 1 : 0;
    s->flops_per_sample = hp.flops_per_sample;
    s->amps_per_sample = hp.amps_per_sample;
    s->device_bytes = (double)plan_device_bytes(hp);
    // shared-memory estimate matching the kernel's layout
    const size_t csz = hp.precision == PW_PREC_FP64 ? 16 : 8;
    auto a16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const int S = hp.hdr.S, P = std::max(hp.hdr.P, 1), K = std::max(hp.hdr.K, 1);
    size_t b = a16(csz << (S * P)) + a16((size_t)K * (csz << (S * (P - 1)))) + a16(4 * K) + a16(csz << S) +
               a16(csz << hp.hdr.max_block) + a16(csz * 32) + a16(csz * 2 * S) + a16(csz / 2 * 32) + a16(hp.hdr.n) * 2 +
               a16((size_t)(hp.hdr.P + 1) * hp.hdr.n) + a16(std::max(1, hp.hdr.n_cost_gates)) +
               a16(hp.hdr.has_segfac ? csz * 2 * (size_t)hp.hdr.n * (hp.hdr.P + 1) : 16) + a16(4 * 18);
    const size_t maxsm = 227 * 1024;
    int gpc = (int)std::max<size_t>(1, std::min<size_t>({8, (size_t)(hp.threads_per_chain == 32 ? 8 : 512 / hp.threads_per_chain),
                                                        maxsm / std::max<size_t>(b, 1)}));
    s->chains_per_cta = gpc;
    s->smem_bytes_per_cta = (int)(b * gpc);
    return PW_OK;
}

int pw_plan_exec_order(const pw_plan* plan, int* order) {
    if (!plan || !order) return set_error(PW_ERR_ARG, "null argument");
    std::copy(plan->hp.exec_order.begin(), plan->hp.exec_order.end(), order);
    return PW_OK;
}

void pw_plan_destroy(pw_plan* plan) {
    if (!plan) return;
    if (plan->d_blob || plan->d_counters || plan->d_stage) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (plan->device >= 0 && plan->device != cur) cudaSetDevice(plan->device);
        if (plan->d_blob) cudaFree(plan->d_blob);
        if (plan->d_counters) cudaFree(plan->d_counters);
        if (plan->d_stage) cudaFree(plan->d_stage);
        if (plan->device >= 0 && plan->device != cur && cur >= 0) cudaSetDevice(cur);
    }
    delete plan;
}

}  // extern "C"

// C ABI of plan construction and inspection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <utility>

#include "pw_internal.h"
#include "smem_layout.h"

using namespace pw;

namespace {

// Threads per chain: at most one per 16-entry tile of the widest frontier
// (32..256), and no more than lets every chain that shared memory admits on
// an SM be resident at once (512 threads of 128 registers per SM). Chains
// then overlap each other's serial phases (resampling, table gathers).
int choose_threads(HostPlan& hp, int requested) {
    if (requested > 0) {
        if (requested % 32 || requested > 256 || (requested & (requested - 1)))
            return -1;
        return requested;
    }
    const long N = 1L << hp.W;
    const long by_work = std::max(32L, std::min(256L, N / 16));
    hp.threads_per_chain = 256;   // (the layout's scratch size depends on it)
    const size_t csz = hp.precision == PW_PREC_FP64 ? 16 : 8;
    const long group = (long)make_layout(hp, csz).group_bytes;
    const long chains = std::max(1L, (228L * 1024) / (group + 1024));
    const long by_regs = std::max(32L, 512L / chains);
    const long t = std::min(by_work, by_regs);
    long pw2 = 32;
    while (pw2 * 2 <= t) pw2 <<= 1;
    return (int)pw2;
}

// A two-qubit gate A = SWAP D with D diagonal (SWAP, iSWAP, fSim(pi/2, phi)):
// A[r][c] != 0 exactly when r is c with its two bits exchanged.
bool swap_class(const Op& op) {
    if (op.kind != OP_GATE || op.qubits.size() != 2) return false;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            const int sc = ((c & 1) << 1) | (c >> 1);
            if ((op.mats[r * 4 + c] != cd(0.0, 0.0)) != (r == sc)) return false;
        }
    return true;
}

// Monomial gates move the chain deterministically (Alg. 1); a SWAP-class gate
// on (a, b) exchanges the contents of two qubits, A|x_a x_b> = D(x)|x_b x_a>.
// Following the qubits' contents on wires instead: the gate becomes its phase
// D on the current wires of (a, b), after which a's content is on b's old wire
// and vice versa, and every later operation acts on the wires its qubits'
// contents are on. Operation positions (the draws' ids) stay the same.
// Returns false (out untouched) when the circuit has no such gate.
bool relabel_swaps(const pw_circuit* c, pw_circuit& out, std::vector<int>& wire_of) {
    bool any = false;
    for (const Op& op : c->ops) any = any || swap_class(op);
    if (!any) return false;
    out.n = c->n;
    out.ops = c->ops;
    wire_of.resize(c->n);
    for (int q = 0; q < c->n; ++q) wire_of[q] = q;
    for (Op& op : out.ops) {
        const bool sw = swap_class(op);
        const int a = op.qubits.size() > 0 ? op.qubits[0] : -1, b = op.qubits.size() > 1 ? op.qubits[1] : -1;
        for (int& q : op.qubits) q = wire_of[q];
        if (sw) {
            std::vector<cd> D(16, cd(0.0, 0.0));
            for (int x = 0; x < 4; ++x) D[x * 4 + x] = op.mats[(((x & 1) << 1) | (x >> 1)) * 4 + x];
            op.mats = D;
            std::swap(wire_of[a], wire_of[b]);
        }
    }
    return true;
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
        pw_circuit relabelled;
        const bool moved = relabel_swaps(c, relabelled, plan->out_wire);
        bool noisy = false;
        for (const Op& op : c->ops) noisy = noisy || op.kind == OP_KRAUS;
        // (with channels, Alg. 2's frame stays on the qubits while the
        // relabelling would carry it with the wires: same distribution, other
        // draws; not offered)
        rc = moved && noisy ? set_error(PW_ERR_UNSUPPORTED, "SWAP-class gates in noisy circuits are not supported")
                            : build_plan(moved ? &relabelled : c, o, plan->hp);
    } catch (const std::bad_alloc&) {
        rc = set_error(PW_ERR_OOM, "allocation failed while planning");
    }
    if (rc) {
        delete plan;
        return rc;
    }
    // (the HBM engine: 128 threads per chain, four chains per SM, whose
    // readouts stream their frontiers from HBM concurrently)
    int tpc = plan->hp.engine == 1 && o.threads_per_chain <= 0 ? 128 : choose_threads(plan->hp, o.threads_per_chain);
    if (tpc < 0) {
        delete plan;
        return set_error(PW_ERR_ARG, "threads_per_chain must be a power of two in 32..256");
    }
    plan->hp.threads_per_chain = tpc;
    {
        // A frontier too large for one CTA's shared memory is spread over a
        // thread-block cluster: each CTA holds 2^wloc entries (128 KB) and the
        // top log2(ctas) index bits (lower legs) select the CTA.
        HostPlan& hp = plan->hp;
        const size_t csz = hp.precision == PW_PREC_FP64 ? 16 : 8;
        const int forced = o.ctas_per_chain;
        if (forced != 0 && forced != 2 && forced != 4 && forced != 8) {
            delete plan;
            return set_error(PW_ERR_ARG, "ctas_per_chain must be 0, 2, 4 or 8");
        }
        if (hp.engine == 1 && forced > 1) {
            delete plan;
            return set_error(PW_ERR_ARG, "ctas_per_chain applies to the on-chip engine only");
        }
        if (hp.engine == 0 && (forced > 1 || make_layout(hp, csz).group_bytes > 200 * 1024) && hp.hdr.P >= 1) {
            int wloc = hp.precision == PW_PREC_FP64 ? 13 : 14;
            if (forced > 1) wloc = hp.W - (forced == 2 ? 1 : forced == 4 ? 2 : 3);
            const int c = hp.W - wloc;
            if (c > 3 || wloc < hp.hdr.S) {
                delete plan;
                return set_error(PW_ERR_TOO_LARGE, "frontier of 2^" + std::to_string(hp.W) +
                                                       " entries needs more than 8 CTAs per chain");
            }
            hp.ctas_per_chain = 1 << c;
            hp.wloc = wloc;
            // one CTA per SM: 512 threads (16 warps, 128 registers each) hide
            // more shared-memory latency than 256
            if (o.threads_per_chain <= 0) hp.threads_per_chain = 512;
            if (make_layout(hp, csz).group_bytes > 227 * 1024) {
                delete plan;
                return set_error(PW_ERR_TOO_LARGE, "per-CTA shared memory exceeds 227 KB");
            }
        }
    }
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
    s->flops_per_amplitude = hp.flops_per_amplitude;
    s->device_bytes = (double)plan_device_bytes(hp);
    // shared memory of the kernel's layout
    const SmemLayout L = make_layout(hp, hp.precision == PW_PREC_FP64 ? 16 : 8);
    const int gpc = hp.ctas_per_chain > 1 ? 1 : groups_per_cta(hp.threads_per_chain, L.group_bytes);
    s->ctas_per_chain = hp.ctas_per_chain;
    s->chains_per_cta = gpc;
    s->smem_bytes_per_cta = L.group_bytes * gpc;
    s->engine = hp.engine == 1 ? PW_ENGINE_HBM : PW_ENGINE_ONCHIP;
    s->gemm = hp.gemm;
    s->dense_tile_bits = hp.dense_k;
    s->dense_passes_per_sample = hp.dense_passes_per_sample;
    s->dense_flops_per_sample = hp.dense_flops_per_sample;
    return PW_OK;
}

int pw_plan_exec_order(const pw_plan* plan, int* order) {
    if (!plan || !order) return set_error(PW_ERR_ARG, "null argument");
    std::copy(plan->hp.exec_order.begin(), plan->hp.exec_order.end(), order);
    return PW_OK;
}

void pw_plan_destroy(pw_plan* plan) {
    if (!plan) return;
    if (plan->d_blob || plan->d_counters || plan->d_stage || plan->d_out_wire || plan->d_in_wire || plan->d_dense ||
        !plan->dense_events.empty()) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (plan->device >= 0 && plan->device != cur) cudaSetDevice(plan->device);
        if (plan->d_blob) dev_free(plan->d_blob);
        if (plan->d_counters) dev_free(plan->d_counters);
        if (plan->d_stage) dev_free(plan->d_stage);
        if (plan->d_out_wire) dev_free(plan->d_out_wire);
        if (plan->d_in_wire) dev_free(plan->d_in_wire);
        if (plan->d_dense) dev_free(plan->d_dense);
        for (void* ev : plan->dense_events) cudaEventDestroy(static_cast<cudaEvent_t>(ev));
        if (plan->device >= 0 && plan->device != cur && cur >= 0) cudaSetDevice(cur);
    }
    delete plan;
}

}  // extern "C"

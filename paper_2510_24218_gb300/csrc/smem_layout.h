// Shared-memory layout of one chain's group in the sampler kernel.
#pragma once

#include <algorithm>
#include <cstddef>

#include "pw_internal.h"

namespace pw {

struct SmemLayout {
    int L, R, Rexp, rowdot, wt, T, sit, tab, stg, ud, uf, pd, cmax, rlp, part, fslot, red, s, x, xmix, gframe, segfac, misc, group_bytes;
};

inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

// Byte offsets of every per-chain array; csz = bytes of one complex value.
inline SmemLayout make_layout(const HostPlan& hp, size_t csz) {
    const DevPlanHeader& h = hp.hdr;
    SmemLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align16(o + bytes);
        return (int)at;
    };
    const int S = h.S, P = std::max(h.P, 1), K = std::max(h.K, 1);
    // the HBM engine keeps the frontier and the environments in HBM (the
    // dense operators are composed by their own kernel); everything after
    // its L region is the chain state saved between launches
    const bool hbm = hp.engine == 1;
    L.L = take(hbm ? 16 : hp.ctas_per_chain > 1 ? csz << hp.wloc : csz << (S * P));   // frontier tensor (this CTA's part)
    L.R = take(hbm ? 16 : (size_t)K * (csz << (S * (P - 1))));    // right environments
    L.Rexp = take(sizeof(int) * K);
    // (one layer in one CTA: every readout collapses straight from L)
    L.rowdot = take(h.P == 1 && hp.ctas_per_chain <= 1 ? 16 : csz << S);
    L.wt = take(csz * ((size_t(1) << (S / 2)) + (size_t(1) << (S - S / 2))));   // readout weights, two halves
    L.T = take(csz << (h.max_block + 1));   // two halves (ping-pong)
    L.sit = take(csz * 4 * (size_t)h.max_block + sizeof(int) * 3 * (size_t)h.max_block);   // block's site data
    L.tab = take(csz * (size_t)std::max(1, h.max_tab));
    L.stg = take(sizeof(DevStage) * (size_t)std::max(1, h.max_stages));
    L.ud = take(sizeof(double) * (size_t)std::max(1, h.n_sampled));
    L.uf = take(sizeof(float) * (size_t)std::max(1, h.n_sampled));
    L.pd = take(hp.ctas_per_chain > 1 ? (size_t)16 << S : 16);   // FP64 partial readout sums
    L.cmax = take(16);
    L.rlp = take(16 * sizeof(void*));   // the cluster ranks' frontier parts
    L.part = take(csz * (size_t)std::max(64, hp.threads_per_chain));   // also the resampling scratch (4 per site)
    L.fslot = take(csz * 2 * S);
    L.red = take((csz / 2) * 32);
    L.s = take(h.n);
    L.x = take(h.n);
    L.xmix = take((size_t)(h.P + 1) * h.n);
    L.gframe = take(std::max(1, h.n_cost_gates));
    L.segfac = take(h.has_segfac ? csz * 2 * (size_t)h.n * (h.P + 1) : 16);
    L.misc = take(sizeof(int) * (2 + 16 + 2));
    L.group_bytes = (int)align16(o);
    return L;
}

// Chains per CTA, chosen to maximise the chains resident on one SM: 228 KB
// of shared memory per SM (1 KB reserved per CTA), at most 512 resident
// threads (128 registers each, the kernel's register budget) and 256 threads per
// CTA.
inline int groups_per_cta(int tpc, int group_bytes) {
    int best = 1, best_chains = 0;
    for (int g = 1; g <= 8 && g * tpc <= 256; ++g) {
        const int by_smem = (228 * 1024) / (g * group_bytes + 1024);
        const int by_threads = 512 / (g * tpc);
        const int ctas = std::min(by_smem, by_threads);
        if (ctas * g > best_chains) {
            best_chains = ctas * g;
            best = g;
        }
    }
    return best;
}

}  // namespace pw

// Shared-memory layout of one chain's group in the sampler kernel.
#pragma once

#include <algorithm>
#include <cstddef>

#include "pw_internal.h"

namespace pw {

struct SmemLayout {
    int L, R, Rexp, rowdot, T, tab, part, fslot, red, s, x, xmix, gframe, segfac, misc, group_bytes;
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
    L.L = take(csz << (S * P));                        // frontier tensor
    L.R = take((size_t)K * (csz << (S * (P - 1))));    // right environments
    L.Rexp = take(sizeof(int) * K);
    L.rowdot = take(csz << S);
    L.T = take(csz << h.max_block);
    L.tab = take(csz * (size_t)std::max(1, h.max_tab));
    L.part = take(csz * 256);
    L.fslot = take(csz * 2 * S);
    L.red = take((csz / 2) * 32);
    L.s = take(h.n);
    L.x = take(h.n);
    L.xmix = take((size_t)(h.P + 1) * h.n);
    L.gframe = take(std::max(1, h.n_cost_gates));
    L.segfac = take(h.has_segfac ? csz * 2 * (size_t)h.n * (h.P + 1) : 16);
    L.misc = take(sizeof(int) * (2 + 16));
    L.group_bytes = (int)align16(o);
    return L;
}

// Chains per CTA: at most 256 threads per CTA (the kernel's launch bounds),
// and enough shared memory left for 3 CTAs per SM when possible.
inline int groups_per_cta(int tpc, int group_bytes) {
    const int maxsm = 227 * 1024;
    return std::max(1, std::min({8, 256 / tpc, (maxsm / 3) / std::max(1, group_bytes)}));
}

}  // namespace pw

// Contraction-plan builder.
//
// The amplitudes the sampler needs at a one-qubit gate of layer m (Alg. 1,
// amp(C_t, y) = <y s_rest| C_t |0^n>) are contractions of the circuit's
// tensor network in which diagonal gates identify legs (App. A): every qubit
// carries a column of wire segments z^0 .. z^m (z^j after the j-th non-diagonal
// gate), cost gates of section j+1 couple segments z^j of two qubits, and the
// one-qubit gates couple z^j to z^{j-1}. For QAOA this is the graph times a
// path of p vertices (App. A).
//
// At layer m the qubits already resampled in this layer carry legs
// z^0..z^{m-1} summed (their z^m is fixed to the new bit), the others carry
// z^0..z^{m-2} summed (z^{m-1} fixed to the current bit). The plan sweeps the
// qubits in an order pi, in blocks:
//   * forward: a frontier tensor L over the legs of the "live" sites (absorbed
//     and still adjacent to unabsorbed sites, or not yet resampled) absorbs the
//     sites of one block, eliminating resampled sites whose neighbours are all
//     absorbed;
//   * backward: at the start of the layer the sites are absorbed in reverse
//     (their top segments fixed to the current bits), which caches one right
//     environment R_k per block over the lower legs of the frontier sites;
//   * readout: T(tops of the block sites) = sum L * R_k * (cross-edge factors of
//     the top segments); the block's sites are then resampled one by one from T.
// The same slot layout serves both directions: slot j holds a site's lower legs
// at bits j*(m-1)+l and its top leg at bit S*(m-1)+j.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <set>
#include <tuple>

#include "pw_internal.h"

namespace pw {

bool lsm_factor(const cd* E, int m, cd* M0, cd* M1);

namespace {

enum EvType { EV_SUMOUT, EV_REPLACE, EV_EXPAND, EV_EDGE, EV_SITE };
struct Event {
    int type, u, v, slot, slot2;   // EV_EDGE: u = new site v, v = live site w, slot/slot2 their slots
};

struct Layered {
    int n = 0, P = 0;
    std::vector<std::vector<int>> mixer_ops;   // [P+1] op ids in circuit order
    std::vector<int> mixer_op_of;              // [(P+1)*n]
    std::vector<std::vector<int>> sections;    // [P+2], sections[m] m = 1..P+1
};

// FP32 copy of a complex FP64 constant. Among the pairs within one unit in
// the last place (per part) of the nearest pair, and no farther from v than
// one unit of the larger part, take the one whose modulus is closest to |v|
// (ties: the nearest). The same rounded constants act at every site of a
// sweep, so their modulus errors would add up coherently over hundreds of
// sites (a common drift of the amplitudes' size); their phase errors stay
// those of a near-nearest rounding, and conjugate constants keep conjugate
// copies. Parts that are exactly zero stay zero.
void round_c32(cd v, float& re, float& im) {
    const float a0 = (float)v.real(), b0 = (float)v.imag();
    re = a0;
    im = b0;
    if (!std::isfinite(a0) || !std::isfinite(b0)) return;
    const double mod = std::abs(v);
    const double ulp = std::max(std::fabs((double)std::nextafter(a0, INFINITY) - a0),
                                std::fabs((double)std::nextafter(b0, INFINITY) - b0));
    double best_m = std::fabs(std::hypot((double)a0, (double)b0) - mod), best_d = std::abs(cd(a0, b0) - v);
    for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j) {
            if ((i && v.real() == 0.0) || (j && v.imag() == 0.0)) continue;
            const float a = i < 0 ? std::nextafter(a0, -INFINITY) : i > 0 ? std::nextafter(a0, INFINITY) : a0;
            const float b = j < 0 ? std::nextafter(b0, -INFINITY) : j > 0 ? std::nextafter(b0, INFINITY) : b0;
            const double d = std::abs(cd(a, b) - v);
            if (d > ulp) continue;
            const double m = std::fabs(std::hypot((double)a, (double)b) - mod);
            if (m < best_m || (m == best_m && d < best_d)) {
                best_m = m;
                best_d = d;
                re = a;
                im = b;
            }
        }
}

int parse_layers(const pw_circuit* c, Layered& L) {
    const int n = c->n;
    L.n = n;
    std::vector<int> pending, deferred;
    std::vector<char> done(n, 0);
    int cur = -1, cur_count = 0;
    for (int id = 0; id < (int)c->ops.size(); ++id) {
        const Op& op = c->ops[id];
        int m = (int)op.qubits.size();
        if (op.kind == OP_GATE) {
            bool diag = is_diagonal(op.mat(0), op.dim());
            if (!diag && m == 2)
                return set_error(PW_ERR_UNSUPPORTED, "non-diagonal two-qubit gates are not supported by this plan family");
            if (!diag) {
                int q = op.qubits[0];
                if (cur >= 0 && cur_count < n) {
                    if (done[q]) return set_error(PW_ERR_UNSUPPORTED, "qubit repeated inside a one-qubit gate layer");
                } else {
                    if (cur == -1 && !pending.empty())
                        return set_error(PW_ERR_UNSUPPORTED, "operations before the first one-qubit gate layer");
                    ++cur;
                    L.mixer_ops.emplace_back();
                    if (cur >= 1) L.sections.push_back(pending);
                    pending.clear();
                    std::fill(done.begin(), done.end(), 0);
                    cur_count = 0;
                }
                done[q] = 1;
                ++cur_count;
                L.mixer_ops[cur].push_back(id);
                if (cur_count == n) {   // layer complete: the ops moved past it open the next section
                    pending = deferred;
                    deferred.clear();
                }
                continue;
            }
        }
        // diagonal gate or channel
        if (cur < 0) return set_error(PW_ERR_UNSUPPORTED, "operations before the first one-qubit gate layer");
        if (cur_count < n) {
            // inside a one-qubit layer: it commutes with the layer's gates on
            // other qubits (and resampling a qubit leaves the others' bits
            // alone), so it moves past the layer when all its qubits already
            // had their gate, or before it when none did
            int nd = 0;
            for (int q : op.qubits) nd += done[q] ? 1 : 0;
            if (nd == m) {
                deferred.push_back(id);
                continue;
            }
            if (nd == 0 && cur >= 1) {
                L.sections.back().push_back(id);
                continue;
            }
            return set_error(PW_ERR_UNSUPPORTED, "a diagonal gate or channel inside a one-qubit gate layer couples "
                                                 "qubits before and after their gate");
        }
        pending.push_back(id);
    }
    if (cur < 0) return set_error(PW_ERR_UNSUPPORTED, "circuit has no layer of one-qubit gates");
    if (cur_count < n) return set_error(PW_ERR_UNSUPPORTED, "last one-qubit gate layer is incomplete");
    L.P = cur;
    // sections[0] unused; sections[m] between mixer m-1 and m; sections[P+1] final
    std::vector<std::vector<int>> secs(L.P + 2);
    for (int m = 1; m <= L.P; ++m) secs[m] = L.sections[m - 1];
    secs[L.P + 1] = pending;
    L.sections = secs;
    L.mixer_op_of.assign((size_t)(L.P + 1) * n, -1);
    for (int m = 0; m <= L.P; ++m)
        for (int id : L.mixer_ops[m]) L.mixer_op_of[(size_t)m * n + c->ops[id].qubits[0]] = id;
    return PW_OK;
}

// ------------------------------------------------------------------ sweep
struct Sweep {
    const std::vector<std::vector<int>>* adj = nullptr;
    std::vector<int> blk, slot, unabs;
    std::vector<int> live;
    std::vector<char> slot_used;
    int peak = 0;
    int nslots = 0;

    void init(const std::vector<std::vector<int>>& a) {
        adj = &a;
        int n = (int)a.size();
        blk.assign(n, -1);
        slot.assign(n, -1);
        unabs.resize(n);
        for (int i = 0; i < n; ++i) unabs[i] = (int)a[i].size();
        live.clear();
        slot_used.clear();
        peak = 0;
        nslots = 0;
    }
    int alloc() {
        for (int j = 0; j < (int)slot_used.size(); ++j)
            if (!slot_used[j]) { slot_used[j] = 1; return j; }
        slot_used.push_back(1);
        nslots = std::max(nslots, (int)slot_used.size());
        return (int)slot_used.size() - 1;
    }
    void release(int u) {
        slot_used[slot[u]] = 0;
        live.erase(std::find(live.begin(), live.end(), u));
    }
    bool adjacent(int a, int b) const {
        const auto& v = (*adj)[a];
        return std::find(v.begin(), v.end(), b) != v.end();
    }
    void absorb_block(const std::vector<int>& sites, int k, std::vector<Event>* ev) {
        // resampled sites whose neighbours are all absorbed leave the frontier
        std::vector<int> cp = live;
        for (int u : cp)
            if (blk[u] < k && unabs[u] == 0) {
                if (ev) ev->push_back({EV_SUMOUT, u, -1, slot[u], -1});
                release(u);
            }
        for (int v : sites) {
            blk[v] = k;
            for (int w : (*adj)[v]) --unabs[w];
            std::vector<int> elig;
            for (int u : live)
                if (blk[u] < k && unabs[u] == 0) elig.push_back(u);
            int ustar = elig.empty() ? -1 : elig[0];
            if (ustar >= 0) {
                slot[v] = slot[ustar];
                if (ev) ev->push_back({EV_REPLACE, ustar, v, slot[v], -1});
                live.erase(std::find(live.begin(), live.end(), ustar));
            } else {
                slot[v] = alloc();
                if (ev) ev->push_back({EV_EXPAND, -1, v, slot[v], -1});
            }
            live.push_back(v);
            peak = std::max(peak, (int)live.size());
            for (int w : live)
                if (w != v && adjacent(v, w) && ev) ev->push_back({EV_EDGE, v, w, slot[v], slot[w]});
            if (ev) ev->push_back({EV_SITE, -1, v, slot[v], -1});
            for (size_t i = 1; i < elig.size(); ++i) {
                if (ev) ev->push_back({EV_SUMOUT, elig[i], -1, slot[elig[i]], -1});
                release(elig[i]);
            }
        }
    }
};

int width_singletons(const std::vector<std::vector<int>>& adj, const std::vector<int>& order, double* cost) {
    Sweep s;
    s.init(adj);
    double c = 0;
    for (int k = 0; k < (int)order.size(); ++k) {
        s.absorb_block({order[k]}, k, nullptr);
        c += std::ldexp(1.0, std::min(60, (int)s.live.size()));
    }
    if (cost) *cost = c;
    return s.nslots;
}

std::vector<std::vector<int>> greedy_blocks(const std::vector<std::vector<int>>& adj, const std::vector<int>& order,
                                            int target, int max_block) {
    Sweep s;
    s.init(adj);
    std::vector<std::vector<int>> blocks;
    std::vector<int> cur;
    Sweep at_start = s;
    for (int v : order) {
        std::vector<int> trial = cur;
        trial.push_back(v);
        Sweep t = at_start;
        t.absorb_block(trial, (int)blocks.size(), nullptr);
        if (cur.empty() || ((int)trial.size() <= max_block && t.nslots <= target)) {
            cur = trial;
            continue;
        }
        at_start.absorb_block(cur, (int)blocks.size(), nullptr);
        blocks.push_back(cur);
        cur = {v};
    }
    if (!cur.empty()) blocks.push_back(cur);
    return blocks;
}

std::vector<int> bfs_order(const std::vector<std::vector<int>>& adj, int start) {
    int n = (int)adj.size();
    std::vector<int> order, seen(n, 0);
    for (int s0 = -1; s0 < n; ++s0) {   // roots: start, then every vertex in turn
        const int s = s0 < 0 ? start : s0;
        if (seen[s]) continue;
        std::vector<int> q{s};
        seen[s] = 1;
        for (size_t h = 0; h < q.size(); ++h) {
            order.push_back(q[h]);
            std::vector<int> nb = adj[q[h]];
            std::sort(nb.begin(), nb.end());
            for (int w : nb)
                if (!seen[w]) { seen[w] = 1; q.push_back(w); }
        }
    }
    return order;
}

// Greedy: repeatedly absorb the vertex that leaves the fewest live sites.
std::vector<int> greedy_order(const std::vector<std::vector<int>>& adj, int start) {
    int n = (int)adj.size();
    std::vector<int> order;
    std::vector<char> absorbed(n, 0);
    std::vector<int> unabs(n), live_flag(n, 0);
    for (int i = 0; i < n; ++i) unabs[i] = (int)adj[i].size();
    int live = 0;
    auto take = [&](int v) {
        absorbed[v] = 1;
        order.push_back(v);
        live_flag[v] = 1;
        ++live;
        for (int w : adj[v]) {
            --unabs[w];
            if (absorbed[w] && unabs[w] == 0 && live_flag[w]) { live_flag[w] = 0; --live; }
        }
        if (unabs[v] == 0) { live_flag[v] = 0; --live; }
    };
    take(start);
    while ((int)order.size() < n) {
        int best = -1;
        long bscore = 0;
        for (int v = 0; v < n; ++v) {
            if (absorbed[v]) continue;
            bool touches = false;
            for (int w : adj[v]) touches |= (bool)absorbed[w];
            if (!touches && best >= 0) continue;
            int delta = 1;
            int nabs = 0;
            for (int w : adj[v])
                if (absorbed[w]) {
                    ++nabs;
                    if (unabs[w] == 1 && live_flag[w]) --delta;
                }
            if (unabs[v] - nabs == 0) --delta;
            long score = (long)delta * 1000 - nabs;
            if (!touches) score += 100000;
            if (best < 0 || score < bscore) { best = v; bscore = score; }
        }
        take(best);
    }
    return order;
}

// Group consecutive micro-ops into tiled passes: the 2x2 matrices of a pass
// act on at most 4 distinct bits (its tile), at most 8 stages per pass, and
// consecutive diagonal/scalar ops merge into one stage while their bits number
// at most 5. Returns the table entries of the range; *nst gets its stages.
int fuse_range(HostPlan& hp, int b, int e, int* nst_out) {
    int tab = 0;
    int i = b;
    const int st0 = (int)hp.stages.size();
    while (i < e) {
        DevFused f{};
        f.st_begin = (int)hp.stages.size();
        std::vector<int> tiles;
        std::vector<std::vector<int>> sbits;   // per stage: diagonal bits
        while (i < e) {
            const DevMicroOp& o = hp.micro[i];
            if (o.kind == MK_MAT1) {
                int bit = o.bits[0];
                auto it = std::find(tiles.begin(), tiles.end(), bit);
                int k;
                if (it == tiles.end()) {
                    if (tiles.size() == 4) break;
                    tiles.push_back(bit);
                    k = (int)tiles.size() - 1;
                } else {
                    k = (int)(it - tiles.begin());
                }
                if (f.nst == 8) break;
                DevStage st{};
                st.type = ST_MAT;
                st.arg = (uint8_t)k;
                st.op_begin = i;
                st.op_end = i + 1;
                {
                    const int rc = hp.micro[i].recipe;
                    st.form = rc == RC_EXPAND ? MF_EXPAND : (rc == RC_SUMOUT1 || rc == RC_SUMOUT_MIX) ? MF_ROW0 : MF_GENERAL;
                }
                hp.stages.push_back(st);
                sbits.emplace_back();
                ++f.nst;
                ++i;
                continue;
            }
            bool merged = false;
            if (f.nst > 0 && hp.stages.back().type == ST_DIAG) {
                std::vector<int> u = sbits.back();
                for (int j = 0; j < o.nbits; ++j)
                    if (std::find(u.begin(), u.end(), (int)o.bits[j]) == u.end()) u.push_back(o.bits[j]);
                if (u.size() <= 5) {
                    sbits.back() = u;
                    hp.stages.back().op_end = i + 1;
                    merged = true;
                }
            }
            if (!merged) {
                if (f.nst == 8) break;
                DevStage st{};
                st.type = ST_DIAG;
                st.op_begin = i;
                st.op_end = i + 1;
                hp.stages.push_back(st);
                std::vector<int> u;
                for (int j = 0; j < o.nbits; ++j)
                    if (std::find(u.begin(), u.end(), (int)o.bits[j]) == u.end()) u.push_back(o.bits[j]);
                sbits.push_back(u);
                ++f.nst;
            }
            ++i;
        }
        f.ntb = (uint8_t)tiles.size();
        for (size_t k = 0; k < tiles.size(); ++k) f.tbits[k] = (uint8_t)tiles[k];
        for (int s = 0; s < f.nst; ++s) {
            DevStage& st = hp.stages[f.st_begin + s];
            for (int k = 0; k < 4; ++k) {
                st.tpos[k] = 0xFF;
                if (st.type == ST_DIAG && k < (int)tiles.size())
                    for (size_t j = 0; j < sbits[s].size(); ++j)
                        if (sbits[s][j] == tiles[k]) st.tpos[k] = (uint8_t)j;
            }
        }
        for (int s = 0; s < f.nst; ++s) {
            DevStage& st = hp.stages[f.st_begin + s];
            st.tab_off = tab;
            if (st.type == ST_MAT) {
                tab += 4;
                continue;
            }
            const std::vector<int>& db = sbits[s];
            st.arg = (uint8_t)db.size();
            for (size_t j = 0; j < db.size(); ++j) st.dbits[j] = (uint8_t)db[j];
            tab += 1 << db.size();
            for (int k = st.op_begin; k < st.op_end; ++k) {
                DevMicroOp& o = hp.micro[k];
                for (int j = 0; j < o.nbits; ++j)
                    o.fpos[j] = (uint8_t)(std::find(db.begin(), db.end(), (int)o.bits[j]) - db.begin());
            }
        }
        hp.fused.push_back(f);
    }
    *nst_out = (int)hp.stages.size() - st0;
    return tab;
}

// Group the micro-ops [b, e) of a forward block program of a dense layer into
// dense passes (executed as GEMMs on the HBM-resident frontier): the 2x2
// matrices of a pass act on at most kd distinct bits, its tile (padded to
// exactly kd bits with free high bits: the operator is the identity on them);
// diagonal factors whose bits all lie in the tile are composed into the
// pass's dense operator in program order; diagonal factors that also read
// other bits are deferred to the pass's epilogue, which is exact because they
// commute with every later matrix of the pass that does not act on one of
// their bits (a matrix that would ends the pass first). At most four deferred
// factors, each over at most five bits, per pass. Stage tables are laid out
// as in fuse_range (a matrix 4 entries, a diagonal 2^bits).
int fuse_dense(HostPlan& hp, int b, int e, int kd, int W, int* nst_out) {
    int tab = 0;
    int i = b;
    const int st0 = (int)hp.stages.size();
    auto uniq_bits = [&](const DevMicroOp& o) {
        std::vector<int> u;
        for (int j = 0; j < o.nbits; ++j)
            if (std::find(u.begin(), u.end(), (int)o.bits[j]) == u.end()) u.push_back(o.bits[j]);
        return u;
    };
    while (i < e) {
        DevFused f{};
        f.st_begin = (int)hp.stages.size();
        std::vector<int> tiles;
        std::vector<std::vector<int>> sbits;   // per stage: diagonal bits
        std::vector<char> sepi;                // per stage: deferred to the epilogue
        int n_epi = 0;
        while (i < e) {
            const DevMicroOp& o = hp.micro[i];
            const int nst = (int)sbits.size();
            if (nst == 250) break;
            if (o.kind == MK_MAT1) {
                const int bit = o.bits[0];
                bool blocked = false;
                for (int s2 = 0; s2 < nst; ++s2)
                    if (sepi[s2] && std::find(sbits[s2].begin(), sbits[s2].end(), bit) != sbits[s2].end()) blocked = true;
                if (blocked) break;
                auto it = std::find(tiles.begin(), tiles.end(), bit);
                int k;
                if (it == tiles.end()) {
                    if ((int)tiles.size() == kd) break;
                    tiles.push_back(bit);
                    k = (int)tiles.size() - 1;
                } else {
                    k = (int)(it - tiles.begin());
                }
                DevStage st{};
                st.type = ST_MAT;
                st.arg = (uint8_t)k;
                st.op_begin = i;
                st.op_end = i + 1;
                const int rc = o.recipe;
                st.form = rc == RC_EXPAND ? MF_EXPAND : (rc == RC_SUMOUT1 || rc == RC_SUMOUT_MIX) ? MF_ROW0 : MF_GENERAL;
                hp.stages.push_back(st);
                sbits.emplace_back();
                sepi.push_back(0);
                ++i;
                continue;
            }
            const std::vector<int> X = uniq_bits(o);
            // a factor reading bits outside the tile takes them into the tile
            // while it has room (they would otherwise be padding): it is then
            // composed into the operator, and later matrices on those bits
            // can join the pass
            {
                std::vector<int> add;
                for (int x : X)
                    if (std::find(tiles.begin(), tiles.end(), x) == tiles.end()) add.push_back(x);
                if (!add.empty() && (int)(tiles.size() + add.size()) <= kd) {
                    bool free_bits = true;   // (no deferred factor may read a bit the tile takes)
                    for (int s2 = 0; s2 < nst; ++s2)
                        if (sepi[s2])
                            for (int x : add)
                                if (std::find(sbits[s2].begin(), sbits[s2].end(), x) != sbits[s2].end()) free_bits = false;
                    if (free_bits) tiles.insert(tiles.end(), add.begin(), add.end());
                }
            }
            bool inside = true;
            for (int x : X) inside = inside && std::find(tiles.begin(), tiles.end(), x) != tiles.end();
            // merge into the previous stage: a diagonal of the same kind, at most 5 bits
            if (nst > 0 && hp.stages.back().type == ST_DIAG && (bool)sepi.back() == !inside) {
                std::vector<int> u = sbits.back();
                for (int x : X)
                    if (std::find(u.begin(), u.end(), x) == u.end()) u.push_back(x);
                if (u.size() <= 5) {
                    sbits.back() = u;
                    hp.stages.back().op_end = i + 1;
                    ++i;
                    continue;
                }
            }
            if (!inside && n_epi == 4) break;
            DevStage st{};
            st.type = ST_DIAG;
            st.op_begin = i;
            st.op_end = i + 1;
            st.epi = inside ? 0 : 1;
            hp.stages.push_back(st);
            sbits.push_back(X);
            sepi.push_back(inside ? 0 : 1);
            if (!inside) ++n_epi;
            ++i;
        }
        // pad the tile with free high bits
        for (int bit = W - 1; (int)tiles.size() < kd && bit >= 0; --bit)
            if (std::find(tiles.begin(), tiles.end(), bit) == tiles.end()) tiles.push_back(bit);
        f.ntb = (uint8_t)kd;
        for (int k = 0; k < kd; ++k) f.tbits[k] = (uint8_t)tiles[k];
        f.nst = (uint8_t)sbits.size();
        for (int s2 = 0; s2 < f.nst; ++s2) {
            DevStage& st = hp.stages[f.st_begin + s2];
            for (int k = 0; k < 4; ++k) st.tpos[k] = 0xFF;
            st.tab_off = tab;
            if (st.type == ST_MAT) {
                tab += 4;
                continue;
            }
            const std::vector<int>& db = sbits[s2];
            st.arg = (uint8_t)db.size();
            for (size_t j = 0; j < db.size(); ++j) st.dbits[j] = (uint8_t)db[j];
            tab += 1 << db.size();
            for (int k = st.op_begin; k < st.op_end; ++k) {
                DevMicroOp& o = hp.micro[k];
                for (int j = 0; j < o.nbits; ++j)
                    o.fpos[j] = (uint8_t)(std::find(db.begin(), db.end(), (int)o.bits[j]) - db.begin());
            }
        }
        hp.fused.push_back(f);
    }
    *nst_out = (int)hp.stages.size() - st0;
    return tab;
}

// ---------------------------------------------------------------------------
// Host precompute of the tables of noiseless plans. Without channels the only
// chain-dependent inputs of a stage's table are the current bits of at most a
// few qubits (the top weight A_m[s_u][.] of an eliminated site, or a fixed top
// segment in the backward sweep); every variant of those bits is evaluated
// here in FP64 once, and the kernel only gathers. Scalar factors (RC_CONST_EDGES)
// are left out: they only change the overall scale of the amplitudes.
struct HostEval {
    const HostPlan& hp;
    std::vector<cd> segfac;   // [n][P+1][2] static one-qubit diagonal factors
    int n, P;
    const int* sq;            // qubit -> position in deps, -1 if not a dependency
    int var;                  // variant bits

    int sbit(int q) const { return sq[q] >= 0 ? (var >> sq[q]) & 1 : 0; }
    cd mix(int m, int q, int o, int i) const {
        const double* d = hp.mix_d.data() + ((size_t)m * n + q) * 8 + 2 * ((o << 1) | i);
        return cd(d[0], d[1]);
    }
    cd gate(int g, int a0, int a1) const {
        const DevCostGate& G = hp.cost_gates[g];
        int idx = a0 | (a1 << 1);
        return cd(G.d[2 * idx], G.d[2 * idx + 1]);
    }
    cd gpair(int g, int qa, int va, int vb) const {
        return hp.cost_gates[g].q0 == qa ? gate(g, va, vb) : gate(g, vb, va);
    }
    cd entry(const DevMicroOp& o, int e) const {
        const int32_t* gref = hp.gate_refs.data();
        switch (o.recipe) {
            case RC_EXPAND: return (e & 1) == 0 ? 1.0 : 0.0;
            case RC_SUMOUT1: return (e >> 1) == 0 ? 1.0 : 0.0;
            case RC_SUMOUT_MIX: return (e >> 1) == 0 ? mix(o.layer, o.qa, sbit(o.qa), e & 1) : cd(0.0);
            case RC_REPLACE: {
                int aout = e >> 1, ain = e & 1;
                cd v = o.layer >= 0 ? mix(o.layer, o.qa, sbit(o.qa), ain) : cd(1.0);
                for (int i = 0; i < o.gcount; ++i) v *= gpair(gref[o.glist + i], o.qa, ain, aout);
                return v;
            }
            case RC_BREPLACE: {
                int aout = e >> 1, ain = e & 1;
                cd v = 1.0;
                for (int i = 0; i < o.gcount; ++i) v *= gpair(gref[o.glist + i], o.qa, aout, ain);
                return v;
            }
            case RC_EDGE: {
                cd v = 1.0;
                for (int i = 0; i < o.gcount; ++i) v *= gpair(gref[o.glist + i], o.qa, e & 1, (e >> 1) & 1);
                return v;
            }
            case RC_SITE: {
                int q = o.qa, nseg = o.layer, z[8];
                for (int l = 0; l < nseg; ++l) z[l] = (e >> l) & 1;
                if (o.fixed_top) z[nseg - 1] = sbit(q);
                cd v = mix(0, q, z[0], 0);
                for (int l = 1; l < nseg; ++l) v *= mix(l, q, z[l], z[l - 1]);
                for (int l = 0; l < nseg; ++l) v *= segfac[((size_t)q * (P + 1) + l) * 2 + z[l]];
                return v;
            }
            default: return 1.0;   // RC_CONST_EDGES: scale only
        }
    }
};

void push_var(HostPlan& hp, cd v) {
    hp.vtab_d.push_back(v.real());
    hp.vtab_d.push_back(v.imag());
    float re, im;
    round_c32(v, re, im);
    hp.vtab_f.push_back(re);
    hp.vtab_f.push_back(im);
}

// Group the items of every cost section into waves. Per qubit there are two
// resources: its frame bit x (read by every item on the qubit, written by a
// channel) and its one-qubit factor of the segment (written by one-qubit
// gates and channels). An item goes one wave after the last writer of what it
// reads and after the last reader or writer of what it writes (a factor is
// only read by its own read-modify-write); within a wave the circuit order is
// kept.
void build_cost_waves(HostPlan& hp, int n, int P) {
    hp.cost_waves.clear();
    hp.cost_wave_ranges.assign(P + 3, 0);
    for (int m = 1; m <= P + 1; ++m) {
        hp.cost_wave_ranges[m] = (int)hp.cost_waves.size();
        const int b = hp.cost_ranges[m], e = hp.cost_ranges[m + 1];
        std::vector<int> wx(n, -1), rx(n, -1), wf(n, -1);
        std::vector<int> wave(e - b);
        int nw = 0;
        for (int it = b; it < e; ++it) {
            const DevCostItem ci = hp.cost_items[it];
            int qs[2], nq = 0;
            bool writes_x = false, writes_f = false;
            if (ci.kind == CI_CHANNEL) {
                const DevChannel& c = hp.channels[ci.idx];
                for (int i = 0; i < c.nq; ++i) qs[nq++] = c.q[i];
                writes_x = writes_f = true;
            } else {
                const DevCostGate& g = hp.cost_gates[ci.idx];
                qs[nq++] = g.q0;
                if (g.q1 >= 0) qs[nq++] = g.q1;
                writes_f = ci.kind == CI_GATE1;
            }
            int w = 0;
            for (int i = 0; i < nq; ++i) {
                const int q = qs[i];
                w = std::max(w, wx[q] + 1);
                if (writes_x) w = std::max(w, rx[q] + 1);
                if (writes_f) w = std::max(w, wf[q] + 1);
            }
            for (int i = 0; i < nq; ++i) {
                const int q = qs[i];
                rx[q] = std::max(rx[q], w);
                if (writes_x) wx[q] = w;
                if (writes_f) wf[q] = w;
            }
            wave[it - b] = w;
            nw = std::max(nw, w + 1);
        }
        std::vector<int> idx(e - b);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return wave[x] < wave[y]; });
        std::vector<DevCostItem> sorted(e - b);
        for (int i = 0; i < e - b; ++i) sorted[i] = hp.cost_items[b + idx[i]];
        std::copy(sorted.begin(), sorted.end(), hp.cost_items.begin() + b);
        for (int w = 0, i = 0; w < nw; ++w) {
            hp.cost_waves.push_back(b + i);
            while (i < e - b && wave[idx[i]] == w) ++i;
        }
    }
    hp.cost_wave_ranges[P + 2] = (int)hp.cost_waves.size();
    hp.cost_waves.push_back((int)hp.cost_items.size());
}

// Variant tables of every stage and live slot, evaluated in FP64. For a noisy
// plan they describe a clean chain: every Kraus draw so far took operator 0
// (identity part of a Pauli channel, E0 of damping), so the frame is zero and
// each segment carries the fixed factors of those operators; the kernel uses
// them only while its chain is clean. The segment factors are kept for the
// chain that leaves that state.
void precompute_tables(HostPlan& hp) {
    const int n = hp.hdr.n, P = hp.hdr.P;
    HostEval ev{hp, std::vector<cd>((size_t)n * (P + 1) * 2, cd(1.0)), n, P, nullptr, 0};
    for (int m = 1; m <= P; ++m)
        for (int it = hp.cost_ranges[m]; it < hp.cost_ranges[m + 1]; ++it) {
            const DevCostItem ci = hp.cost_items[it];
            if (ci.kind == CI_GATE1) {
                const DevCostGate& G = hp.cost_gates[ci.idx];
                for (int b = 0; b < 2; ++b) ev.segfac[((size_t)G.q0 * (P + 1) + (m - 1)) * 2 + b] *= cd(G.d[2 * b], G.d[2 * b + 1]);
            } else if (ci.kind == CI_CHANNEL) {
                const DevChannel& c = hp.channels[ci.idx];
                for (int f = 0; f < c.nq; ++f) {
                    const DevKrausFactor& F = hp.factors[c.fac_off + f];   // operator 0
                    for (int b = 0; b < 2; ++b)
                        ev.segfac[((size_t)F.q * (P + 1) + (m - 1)) * 2 + b] *= cd(F.d[2 * b], F.d[2 * b + 1]);
                }
            }
        }
    if (hp.hdr.has_frame) {
        hp.segdef_d.clear();
        hp.segdef_f.clear();
        for (const cd& v : ev.segfac) {
            hp.segdef_d.push_back(v.real());
            hp.segdef_d.push_back(v.imag());
            float re, im;
            round_c32(v, re, im);
            hp.segdef_f.push_back(re);
            hp.segdef_f.push_back(im);
        }
    }
    std::vector<int> sq(n, -1);
    ev.sq = sq.data();
    auto deps_of = [&](const DevMicroOp& o, std::vector<int>& deps) {
        bool dep = o.recipe == RC_SUMOUT_MIX || (o.recipe == RC_REPLACE && o.layer >= 0) ||
                   (o.recipe == RC_SITE && o.fixed_top);
        if (dep && std::find(deps.begin(), deps.end(), (int)o.qa) == deps.end()) deps.push_back(o.qa);
    };
    for (DevStage& st : hp.stages) {
        std::vector<int> deps;
        for (int k = st.op_begin; k < st.op_end; ++k) deps_of(hp.micro[k], deps);
        if (deps.size() > 4) {
            st.ndep = 0xFF;
            continue;
        }
        st.ndep = (uint8_t)deps.size();
        for (size_t j = 0; j < deps.size(); ++j) {
            st.dep[j] = (int16_t)deps[j];
            sq[deps[j]] = (int)j;
        }
        st.var_off = (int32_t)(hp.vtab_d.size() / 2);
        const int size = st.type == ST_MAT ? 4 : (1 << st.arg);
        for (int v = 0; v < (1 << deps.size()); ++v) {
            ev.var = v;
            for (int e = 0; e < size; ++e) {
                cd val;
                if (st.type == ST_MAT) {
                    val = ev.entry(hp.micro[st.op_begin], e);
                } else {
                    val = 1.0;
                    for (int k = st.op_begin; k < st.op_end; ++k) {
                        const DevMicroOp& o = hp.micro[k];
                        int loc = 0;
                        for (int j = 0; j < o.nbits; ++j) loc |= ((e >> o.fpos[j]) & 1) << j;
                        val *= ev.entry(o, loc);
                    }
                }
                push_var(hp, val);
            }
        }
        for (int q : deps) sq[q] = -1;
    }
    // readout factors of the live slots (layer of each block range)
    for (int m = 1; m <= P; ++m)
        for (int k = 0; k < hp.hdr.K; ++k) {
            const DevBlockRange& br = hp.block_ranges[(size_t)m * hp.hdr.K + k];
            for (int j = br.live_begin; j < br.live_end; ++j) {
                DevLiveSlot& sl = hp.live_slots[j];
                if (sl.q < 0) {
                    sl.ndep = 0;
                    sl.var_off = (int32_t)(hp.vtab_d.size() / 2);
                    push_var(hp, 1.0);
                    push_var(hp, 0.0);
                    continue;
                }
                std::vector<int> deps;
                for (int i = 0; i < sl.dcount; ++i) {
                    const DevCostGate& G = hp.cost_gates[hp.gate_refs[sl.dlist + i]];
                    int w = G.q0 == sl.q ? G.q1 : G.q0;
                    if (std::find(deps.begin(), deps.end(), w) == deps.end()) deps.push_back(w);
                }
                if (sl.role < 0) deps.push_back(sl.q);
                if (deps.size() > 5) {
                    sl.ndep = 0xFF;
                    continue;
                }
                sl.ndep = (int16_t)deps.size();
                for (size_t i = 0; i < deps.size(); ++i) {
                    sl.dep[i] = (int16_t)deps[i];
                    sq[deps[i]] = (int)i;
                }
                sl.var_off = (int32_t)(hp.vtab_d.size() / 2);
                for (int v = 0; v < (1 << deps.size()); ++v) {
                    ev.var = v;
                    for (int top = 0; top < 2; ++top) {
                        cd f = 1.0;
                        for (int i = 0; i < sl.dcount; ++i) {
                            const int g = hp.gate_refs[sl.dlist + i];
                            const DevCostGate& G = hp.cost_gates[g];
                            int w = G.q0 == sl.q ? G.q1 : G.q0;
                            f *= ev.gpair(g, sl.q, top, ev.sbit(w));
                        }
                        if (sl.role < 0) f *= ev.mix(m, sl.q, ev.sbit(sl.q), top);
                        push_var(hp, f);
                    }
                }
                for (int q : deps) sq[q] = -1;
            }
        }
}

}  // namespace

int build_plan(const pw_circuit* c, const pw_plan_opts& opts, HostPlan& hp) {
    if (!c) return set_error(PW_ERR_ARG, "circuit is null");
    Layered L;
    int rc = parse_layers(c, L);
    if (rc) return rc;
    const int n = c->n, P = L.P;
    if (P > 4) return set_error(PW_ERR_UNSUPPORTED, "more than 4 layers after the first are not supported");
    hp = HostPlan();
    hp.precision = opts.precision == PW_PREC_FP64 ? PW_PREC_FP64 : PW_PREC_FP32;
    if (opts.precision != PW_PREC_FP32 && opts.precision != PW_PREC_FP64)
        return set_error(PW_ERR_ARG, "unknown precision");
    const int max_block = opts.max_block > 0 ? std::min(opts.max_block, 10) : 8;

    // ------------------------------------------------ mixers (2x2 per layer, qubit)
    hp.mix_d.assign((size_t)(P + 1) * n * 8, 0.0);
    hp.mix_mono.assign((size_t)(P + 1) * n, 0);
    for (int m = 0; m <= P; ++m)
        for (int q = 0; q < n; ++q) {
            const Op& op = c->ops[L.mixer_op_of[(size_t)m * n + q]];
            for (int i = 0; i < 4; ++i) {
                hp.mix_d[((size_t)m * n + q) * 8 + 2 * i] = op.mats[i].real();
                hp.mix_d[((size_t)m * n + q) * 8 + 2 * i + 1] = op.mats[i].imag();
            }
            hp.mix_mono[(size_t)m * n + q] = is_monomial(op.mat(0), 2) ? 1 : 0;
        }
    // First-layer gates whose entries all have modulus 2^-1/2 (Hadamard-like):
    // in pairs, their entries are stored times sqrt(2) (unit modulus, exact
    // for +-1 and +-i) and the factor 2^-1 per pair goes to the amplitudes'
    // power-of-two exponent. 1/sqrt(2) has no exact FP32 (or FP64) copy, and
    // its rounding error would otherwise act once per qubit on every
    // amplitude (about -7e-6 at 400 qubits in FP32).
    {
        std::vector<int> hq;
        for (int q = 0; q < n; ++q) {
            const double* A = hp.mix_d.data() + (size_t)q * 8;
            bool h = true;
            for (int i = 0; i < 4; ++i)
                h = h && std::fabs(std::hypot(A[2 * i], A[2 * i + 1]) * std::sqrt(2.0) - 1.0) < 1e-14;
            if (h) hq.push_back(q);
        }
        if (hq.size() % 2) hq.pop_back();
        for (int q : hq) {
            double* A = hp.mix_d.data() + (size_t)q * 8;
            for (int i = 0; i < 4; ++i) {
                const double r = std::hypot(A[2 * i], A[2 * i + 1]);
                A[2 * i] /= r;
                A[2 * i + 1] /= r;
            }
        }
        hp.hdr.amp_exp = -(int)hq.size() / 2;
    }
    hp.mix_f.assign(hp.mix_d.size(), 0.0f);
    for (size_t i = 0; i + 1 < hp.mix_d.size(); i += 2)
        round_c32(cd(hp.mix_d[i], hp.mix_d[i + 1]), hp.mix_f[i], hp.mix_f[i + 1]);
    for (int id : L.mixer_ops[0]) {
        hp.mix0_order.push_back(c->ops[id].qubits[0]);
    }
    hp.mix0_opid.assign(n, -1);
    for (int q = 0; q < n; ++q) hp.mix0_opid[q] = L.mixer_op_of[q];

    // ------------------------------------------------ cost sections
    std::vector<std::vector<int>> adj(n);
    std::map<std::tuple<int, int, int>, std::vector<int>> pair_gates;   // (a<b, level) -> cost gates
    std::vector<std::vector<int>> level_gates(std::max(P, 1));
    hp.cost_ranges.assign(P + 3, 0);
    bool has_segfac = false, has_frame = false;
    for (int m = 1; m <= P + 1; ++m) {
        hp.cost_ranges[m] = (int)hp.cost_items.size();
        for (int id : L.sections[m]) {
            const Op& op = c->ops[id];
            if (op.kind == OP_GATE) {
                if (m == P + 1) continue;   // diagonal gates on fixed final segments: constants
                DevCostGate g{};
                g.q0 = (int16_t)op.qubits[0];
                g.q1 = (int16_t)(op.qubits.size() == 2 ? op.qubits[1] : -1);
                g.level = (int16_t)(m - 1);
                int dim = op.dim();
                for (int b = 0; b < 4; ++b) {
                    cd v = b < dim ? op.mats[(size_t)b * dim + b] : cd(1.0, 0.0);
                    g.d[2 * b] = v.real();
                    g.d[2 * b + 1] = v.imag();
                    round_c32(v, g.f[2 * b], g.f[2 * b + 1]);
                }
                int gi = (int)hp.cost_gates.size();
                hp.cost_gates.push_back(g);
                if (g.q1 >= 0) {
                    int a = std::min<int>(g.q0, g.q1), b = std::max<int>(g.q0, g.q1);
                    if (std::find(adj[a].begin(), adj[a].end(), b) == adj[a].end()) {
                        adj[a].push_back(b);
                        adj[b].push_back(a);
                    }
                    pair_gates[{a, b, m - 1}].push_back(gi);
                    level_gates[m - 1].push_back(gi);
                    hp.cost_items.push_back({CI_GATE2, 0, gi});
                } else {
                    has_segfac = true;
                    hp.cost_items.push_back({CI_GATE1, 0, gi});
                }
            } else {
                has_segfac = true;
                has_frame = true;
                DevChannel ch{};
                ch.op_id = id;
                ch.nq = (int16_t)op.qubits.size();
                ch.k = (int16_t)op.k;
                for (int i = 0; i < ch.nq; ++i) ch.q[i] = (int16_t)op.qubits[i];
                ch.cum_off = (int)hp.cum.size();
                ch.fac_off = (int)hp.factors.size();
                int dim = op.dim();
                for (int cb = 0; cb < dim; ++cb) {
                    double acc = 0;
                    for (int i = 0; i < op.k; ++i) {
                        const cd* E = op.mat(i);
                        double p = 0;
                        for (int r = 0; r < dim; ++r) p += std::norm(E[r * dim + cb]);   // Eq. (5)
                        acc += p;
                        hp.cum.push_back(acc);
                    }
                }
                for (int i = 0; i < op.k; ++i) {
                    cd M[2][4];
                    if (!lsm_factor(op.mat(i), ch.nq, M[0], M[1]))
                        return set_error(PW_ERR_NOT_LSM, "Kraus operator is not local-submonomial");
                    for (int f = 0; f < ch.nq; ++f) {
                        DevKrausFactor kf{};
                        kf.q = ch.q[f];
                        const cd* F = M[f];
                        // Alg. 2: M anti-diagonal <=> M sigma_X diagonal and M not diagonal
                        bool diagM = F[1] == cd(0, 0) && F[2] == cd(0, 0);
                        bool diagMX = F[0] == cd(0, 0) && F[3] == cd(0, 0);
                        cd d0, d1;
                        if (diagMX && !diagM) {
                            kf.antidiag = 1;
                            d0 = F[1];   // (M sigma_X)[0][0] = M[0][1]
                            d1 = F[2];   // (M sigma_X)[1][1] = M[1][0]
                        } else {
                            kf.antidiag = 0;
                            d0 = F[0];
                            d1 = F[3];
                        }
                        kf.d[0] = d0.real();
                        kf.d[1] = d0.imag();
                        kf.d[2] = d1.real();
                        kf.d[3] = d1.imag();
                        hp.factors.push_back(kf);
                    }
                }
                int ci = (int)hp.channels.size();
                hp.channels.push_back(ch);
                hp.cost_items.push_back({CI_CHANNEL, 0, ci});
            }
        }
    }
    hp.cost_ranges[P + 2] = (int)hp.cost_items.size();
    hp.noisy = has_frame;
    build_cost_waves(hp, n, P);

    // ------------------------------------------------ sweep order and blocks
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    if (opts.order == PW_ORDER_AUTO && P >= 1) {
        double best_cost = 0;
        int best_w = width_singletons(adj, order, &best_cost);
        std::vector<std::vector<int>> cands;
        std::vector<int> rev(order.rbegin(), order.rend());
        cands.push_back(rev);
        std::vector<int> starts = {0, n - 1};
        std::vector<int> bydeg(n);
        std::iota(bydeg.begin(), bydeg.end(), 0);
        std::stable_sort(bydeg.begin(), bydeg.end(), [&](int a, int b) { return adj[a].size() < adj[b].size(); });
        for (int i = 0; i < std::min(n, 6); ++i) starts.push_back(bydeg[i]);
        for (int i = 0; i < 4; ++i) starts.push_back((int)((long)i * n / 4));
        for (int s : starts) {
            cands.push_back(bfs_order(adj, s));
            if (n <= 2048) cands.push_back(greedy_order(adj, s));
        }
        for (auto& o : cands) {
            std::vector<int> chk = o;   // (every candidate must order every qubit once)
            std::sort(chk.begin(), chk.end());
            bool perm = (int)chk.size() == n;
            for (int i = 0; perm && i < n; ++i) perm = chk[i] == i;
            if (!perm) continue;
            double cst = 0;
            int wdt = width_singletons(adj, o, &cst);
            if (wdt < best_w || (wdt == best_w && cst < best_cost)) {
                best_w = wdt;
                best_cost = cst;
                order = o;
            }
        }
    } else if (opts.order != PW_ORDER_NATURAL && opts.order != PW_ORDER_AUTO) {
        return set_error(PW_ERR_ARG, "unknown order option");
    }
    hp.sweep_order = order;
    int target = width_singletons(adj, order, nullptr);
    hp.blocks = P >= 1 ? greedy_blocks(adj, order, target, max_block) : std::vector<std::vector<int>>{};
    const int K = (int)hp.blocks.size();

    // final simulation with events
    Sweep sw;
    sw.init(adj);
    std::vector<std::vector<Event>> ev(K);
    std::vector<std::vector<std::pair<int, int>>> live_at(K);   // (site, slot) after block k
    for (int k = 0; k < K; ++k) {
        sw.absorb_block(hp.blocks[k], k, &ev[k]);
        for (int u : sw.live) live_at[k].push_back({u, sw.slot[u]});
    }
    const int S = std::max(1, sw.nslots);
    std::vector<int> blk = sw.blk;
    // engine: the frontier in shared memory (one CTA or a cluster of up to 8
    // holds 2^17 FP32 entries), or in HBM with the wide layers' forward passes
    // run as dense GEMMs (FP32 plans)
    if (opts.engine != PW_ENGINE_AUTO && opts.engine != PW_ENGINE_ONCHIP && opts.engine != PW_ENGINE_HBM)
        return set_error(PW_ERR_ARG, "unknown engine");
    if (opts.gemm != PW_GEMM_SPLIT3 && opts.gemm != PW_GEMM_SPLIT2 && opts.gemm != PW_GEMM_BF16 &&
        opts.gemm != PW_GEMM_FP32)
        return set_error(PW_ERR_ARG, "unknown gemm kind");
    if (opts.engine == PW_ENGINE_HBM && hp.precision != PW_PREC_FP32)
        return set_error(PW_ERR_UNSUPPORTED, "the HBM engine runs FP32 plans only");
    const bool hbm = P >= 1 && hp.precision == PW_PREC_FP32 &&
                     (opts.engine == PW_ENGINE_HBM || (opts.engine == PW_ENGINE_AUTO && S * P > 17));
    hp.engine = hbm ? 1 : 0;
    hp.gemm = opts.gemm;
    if (P >= 1 && !hbm && S * P > 24)
        return set_error(PW_ERR_TOO_LARGE, "frontier tensor of 2^" + std::to_string(S * P) +
                                               " entries per chain exceeds the on-chip engine's limit (2^24)");
    if (P >= 1 && hbm && S * P > 30)
        return set_error(PW_ERR_TOO_LARGE, "frontier tensor of 2^" + std::to_string(S * P) +
                                               " entries per chain exceeds the HBM engine's limit (2^30)");
    // dense layers: the forward frontier of layer m has 2^(S m) entries; its
    // passes become GEMMs of 128-row tiles with 2^kd-entry rows
    auto dense_k = [&](int m) { return !hbm ? 0 : S * m >= 14 ? 6 : S * m >= 12 ? 5 : 0; };

    auto gates_between = [&](int a, int b, int level) -> std::vector<int> {
        auto it = pair_gates.find({std::min(a, b), std::max(a, b), level});
        if (it == pair_gates.end()) return {};
        return it->second;
    };
    auto push_glist = [&](const std::vector<int>& g) {
        int off = (int)hp.gate_refs.size();
        hp.gate_refs.insert(hp.gate_refs.end(), g.begin(), g.end());
        return off;
    };

    // ------------------------------------------------ compile per layer
    hp.block_ranges.assign((size_t)(P + 1) * std::max(K, 1), DevBlockRange{});
    int trace_row = 0;
    double flops = 0;
    hp.exec_order.clear();
    for (int id : L.mixer_ops[0]) hp.exec_order.push_back(id);
    hp.exec_layer.assign(c->ops.size(), -1);
    hp.exec_block.assign(c->ops.size(), -1);
    hp.exec_pos.assign(c->ops.size(), -1);
    for (int m = 1; m <= P; ++m) {
        for (int id : L.sections[m]) hp.exec_order.push_back(id);
        const int Wl = S * (m - 1);
        const int Wm = S * m;
        // forward tensor: top leg of slot j at bit j, lower legs above bit S
        auto bitf = [&](int j, int l) { return l == m - 1 ? j : S + j * (m - 1) + l; };
        auto bitb = [&](int j, int l) { return j * (m - 1) + l; };
        auto mk = [&](uint8_t kind, uint8_t rcp, std::initializer_list<int> bits, int qa, int qb, int layer,
                      const std::vector<int>& gl, int fixed_top) {
            DevMicroOp o{};
            o.kind = kind;
            o.recipe = rcp;
            o.nbits = (uint8_t)bits.size();
            int i = 0;
            for (int b : bits) o.bits[i++] = (uint8_t)b;
            o.qa = (int16_t)qa;
            o.qb = (int16_t)qb;
            o.layer = (int16_t)layer;
            o.fixed_top = (uint8_t)fixed_top;
            o.glist = gl.empty() ? 0 : push_glist(gl);
            o.gcount = (int)gl.size();
            hp.micro.push_back(o);
        };
        for (int k = 0; k < K; ++k) {
            DevBlockRange& br = hp.block_ranges[(size_t)m * K + k];
            // forward
            br.fwd_begin = (int)hp.micro.size();
            for (const Event& e : ev[k]) {
                switch (e.type) {
                    case EV_SUMOUT:
                        for (int l = 0; l < m; ++l)
                            mk(MK_MAT1, l == m - 1 ? RC_SUMOUT_MIX : RC_SUMOUT1, {bitf(e.slot, l)}, e.u, -1,
                               l == m - 1 ? m : -1, {}, 0);
                        break;
                    case EV_REPLACE:
                        for (int l = 0; l < m; ++l)
                            mk(MK_MAT1, RC_REPLACE, {bitf(e.slot, l)}, e.u, e.v, l == m - 1 ? m : -1,
                               gates_between(e.u, e.v, l), 0);
                        break;
                    case EV_EXPAND:
                        for (int l = 0; l < m; ++l) mk(MK_MAT1, RC_EXPAND, {bitf(e.slot, l)}, -1, -1, -1, {}, 0);
                        break;
                    case EV_EDGE:
                        for (int l = 0; l < m; ++l) {
                            std::vector<int> gl = gates_between(e.u, e.v, l);
                            if (!gl.empty())
                                mk(MK_DIAG, RC_EDGE, {bitf(e.slot, l), bitf(e.slot2, l)}, e.u, e.v, -1, gl, 0);
                        }
                        break;
                    case EV_SITE: {
                        DevMicroOp o{};
                        std::vector<int> bits;
                        for (int l = 0; l < m; ++l) bits.push_back(bitf(e.slot, l));
                        o.kind = MK_DIAG;
                        o.recipe = RC_SITE;
                        o.nbits = (uint8_t)m;
                        for (int l = 0; l < m; ++l) o.bits[l] = (uint8_t)bits[l];
                        o.qa = (int16_t)e.v;
                        o.qb = -1;
                        o.layer = (int16_t)m;
                        o.fixed_top = 0;
                        hp.micro.push_back(o);
                        break;
                    }
                }
            }
            {
                int mb = br.fwd_begin, me = (int)hp.micro.size();
                br.fwd_begin = (int)hp.fused.size();
                br.fwd_st = (int)hp.stages.size();
                const int kd = dense_k(m);
                br.fwd_tab = kd ? fuse_dense(hp, mb, me, kd, S * m, &br.fwd_nst) : fuse_range(hp, mb, me, &br.fwd_nst);
                br.fwd_end = (int)hp.fused.size();
            }
            // backward (R_k -> R_{k-1}); not needed for k = 0
            br.bwd_begin = br.bwd_end = (int)hp.fused.size();
            br.bwd_tab = 0;
            br.bwd_st = (int)hp.stages.size();
            br.bwd_nst = 0;
            const int bwd_micro_begin = (int)hp.micro.size();
            if (k >= 1) {
                std::vector<int> consts;
                for (int g : level_gates[m - 1]) {
                    int a = hp.cost_gates[g].q0, b = hp.cost_gates[g].q1;
                    if (std::min(blk[a], blk[b]) == k) consts.push_back(g);
                }
                if (!consts.empty()) mk(MK_CONST, RC_CONST_EDGES, {}, -1, -1, -1, consts, 0);
                for (int i = (int)ev[k].size() - 1; i >= 0; --i) {
                    const Event& e = ev[k][i];
                    switch (e.type) {
                        case EV_SITE: {
                            DevMicroOp o{};
                            o.kind = m >= 2 ? MK_DIAG : MK_CONST;
                            o.recipe = RC_SITE;
                            o.nbits = (uint8_t)(m - 1);
                            for (int l = 0; l < m - 1; ++l) o.bits[l] = (uint8_t)bitb(e.slot, l);
                            o.qa = (int16_t)e.v;
                            o.qb = -1;
                            o.layer = (int16_t)m;
                            o.fixed_top = 1;
                            hp.micro.push_back(o);
                            break;
                        }
                        case EV_REPLACE:
                            for (int l = 0; l < m - 1; ++l)
                                mk(MK_MAT1, RC_BREPLACE, {bitb(e.slot, l)}, e.u, e.v, -1, gates_between(e.u, e.v, l), 0);
                            break;
                        case EV_EXPAND:
                            for (int l = 0; l < m - 1; ++l) mk(MK_MAT1, RC_SUMOUT1, {bitb(e.slot, l)}, -1, -1, -1, {}, 0);
                            break;
                        case EV_SUMOUT:
                            for (int l = 0; l < m - 1; ++l) mk(MK_MAT1, RC_EXPAND, {bitb(e.slot, l)}, -1, -1, -1, {}, 0);
                            break;
                        case EV_EDGE:
                            for (int l = 0; l < m - 1; ++l) {
                                std::vector<int> gl = gates_between(e.u, e.v, l);
                                if (!gl.empty())
                                    mk(MK_DIAG, RC_EDGE, {bitb(e.slot, l), bitb(e.slot2, l)}, e.u, e.v, -1, gl, 0);
                            }
                            break;
                    }
                }
                br.bwd_begin = (int)hp.fused.size();
                br.bwd_st = (int)hp.stages.size();
                br.bwd_tab = fuse_range(hp, bwd_micro_begin, (int)hp.micro.size(), &br.bwd_nst);
                br.bwd_end = (int)hp.fused.size();
            }
        }
        // readout metadata and block sites
        for (int k = 0; k < K; ++k) {
            DevBlockRange& br = hp.block_ranges[(size_t)m * K + k];
            br.site_begin = (int)hp.block_sites.size();
            for (int q : hp.blocks[k]) {
                DevBlockSite bs{};
                bs.q = (int16_t)q;
                bs.monomial = hp.mix_mono[(size_t)m * n + q];
                bs.op_id = L.mixer_op_of[(size_t)m * n + q];
                bs.trace_row = bs.monomial ? -1 : trace_row++;
                if (!bs.monomial) hp.row_opid.push_back(bs.op_id);
                hp.block_sites.push_back(bs);
                hp.exec_order.push_back(bs.op_id);
                hp.exec_layer[bs.op_id] = m;
                hp.exec_block[bs.op_id] = k;
                hp.exec_pos[bs.op_id] = (int)(hp.block_sites.size() - 1 - br.site_begin);
            }
            br.site_end = (int)hp.block_sites.size();
            br.live_begin = (int)hp.live_slots.size();
            std::vector<DevLiveSlot> ls(S);
            for (auto& s : ls) { s.q = -1; s.role = -1; s.dlist = 0; s.dcount = 0; }
            for (auto [u, j] : live_at[k]) {
                ls[j].q = (int16_t)u;
                int role = -1;
                for (int i = 0; i < (int)hp.blocks[k].size(); ++i)
                    if (hp.blocks[k][i] == u) role = i;
                ls[j].role = (int16_t)role;
                std::vector<int> dl;
                for (int w : adj[u])
                    if (blk[w] > k)
                        for (int g : gates_between(u, w, m - 1)) dl.push_back(g);
                ls[j].dcount = (int)dl.size();
                ls[j].dlist = dl.empty() ? 0 : push_glist(dl);
            }
            for (auto& s : ls) hp.live_slots.push_back(s);
            br.live_end = (int)hp.live_slots.size();
            br.rmask = 0;
            for (int j = 0; j < S; ++j)
                if (ls[j].q >= 0 && ls[j].role >= 0) {
                    br.rslot[ls[j].role] = (int8_t)j;
                    br.rmask |= 1 << j;
                }
        }
        (void)Wm;
    }
    for (int id : L.sections[P + 1]) hp.exec_order.push_back(id);
    // algorithmic real flops per sample: a general 2x2 on one bit costs 14
    // flops per entry (two complex multiplies and one add), a row-0 one half
    // of that (its other row is zero), an expand none (a copy); the fused
    // diagonal factor 6; the readout's dot product with R_k 8 per entry of L
    auto stage_flops = [&](const DevStage& st) {
        if (st.type != ST_MAT) return 6.0;
        return st.form == MF_EXPAND ? 0.0 : st.form == MF_ROW0 ? 7.0 : 14.0;
    };
    for (int m = 1; m <= P; ++m) {
        double NF = std::ldexp(1.0, S * m), NB = std::ldexp(1.0, S * (m - 1));
        for (int k = 0; k < K; ++k) {
            const DevBlockRange& br = hp.block_ranges[(size_t)m * K + k];
            for (int i = br.fwd_st; i < br.fwd_st + br.fwd_nst; ++i) flops += stage_flops(hp.stages[i]) * NF;
            for (int i = br.bwd_st; i < br.bwd_st + br.bwd_nst; ++i) flops += stage_flops(hp.stages[i]) * NB;
            flops += 8.0 * NF;
        }
    }
    hp.flops_per_sample = flops;
    // dense passes: each a GEMM of 2^(S m) entries x 2^kd complex multiply-adds
    hp.hdr.dense_mask = 0;
    hp.hdr.dense_npass = 0;
    hp.pass_live_in.assign(hp.fused.size(), 0);
    hp.pass_live_out.assign(hp.fused.size(), 0);
    for (int m = 1; m <= P; ++m) {
        const int kd = dense_k(m);
        if (!kd) continue;
        hp.hdr.dense_mask |= 1 << m;
        hp.dense_k = kd;
        // live legs: a 2x2 stage that copies a leg (a new site's leg) makes it
        // live, one whose second row is zero (a leg summed out) makes it dead,
        // any other keeps it live; diagonal factors keep every leg
        uint32_t live = 0;
        for (int k = 0; k < K; ++k) {
            const DevBlockRange& br = hp.block_ranges[(size_t)m * K + k];
            const int np = br.fwd_end - br.fwd_begin;
            hp.hdr.dense_npass = std::max(hp.hdr.dense_npass, np);
            hp.dense_passes_per_sample += np;
            for (int fi = br.fwd_begin; fi < br.fwd_end; ++fi) {
                const DevFused& f = hp.fused[fi];
                hp.pass_live_in[fi] = live;
                for (int s2 = 0; s2 < f.nst; ++s2) {
                    const DevStage& st = hp.stages[f.st_begin + s2];
                    if (st.type != ST_MAT) continue;
                    const uint32_t bit = 1u << f.tbits[st.arg];
                    live = st.form == MF_ROW0 ? live & ~bit : live | bit;
                }
                hp.pass_live_out[fi] = live;
                // the GEMM covers 2^(kd + 7) entries per tile, its tiles the live outer bits
                int rows[7], outer[32];
                const int no = dense_pass_bits(hp, fi, S * m, rows, outer);
                hp.dense_flops_per_sample += std::ldexp(8.0, 2 * kd + 7 + no);
            }
        }
    }
    // the amplitude of the whole circuit contracts only the last layer's
    // forward sweep, up to the block of the last gate
    {
        int kend = K - 1;
        for (auto it = hp.exec_order.rbegin(); it != hp.exec_order.rend(); ++it)
            if (hp.exec_layer[*it] == P) {
                kend = hp.exec_block[*it];
                break;
            }
        const double NF = std::ldexp(1.0, S * P);
        double a = 0.0;
        for (int k = 0; k <= kend && k < K; ++k) {
            const DevBlockRange& br = hp.block_ranges[(size_t)P * K + k];
            for (int i = br.fwd_st; i < br.fwd_st + br.fwd_nst; ++i) a += stage_flops(hp.stages[i]) * NF;
            a += 8.0 * NF;
        }
        hp.flops_per_amplitude = a;
    }
    hp.amps_per_sample = 2.0 * trace_row;
    hp.hdr.n = n;
    hp.hdr.P = P;
    hp.hdr.S = S;
    hp.hdr.K = K;
    hp.hdr.n_ops = (int)c->ops.size();
    hp.hdr.n_cost_gates = (int)hp.cost_gates.size();
    hp.hdr.n_channels = (int)hp.channels.size();
    hp.hdr.n_sampled = trace_row;
    hp.hdr.max_block = 1;
    for (auto& b : hp.blocks) hp.hdr.max_block = std::max<int>(hp.hdr.max_block, (int)b.size());
    hp.hdr.has_segfac = has_segfac ? 1 : 0;
    hp.hdr.has_frame = has_frame ? 1 : 0;
    hp.hdr.words = (n + 63) / 64;
    // tables: precomputed for noiseless plans and for the clean chains of a
    // noisy plan (possible when no Kraus operator 0 flips the frame); chains
    // with a frame or other Kraus factors build theirs
    for (auto& st : hp.stages) st.ndep = 0xFF;
    for (auto& sl : hp.live_slots) sl.ndep = 0xFF;
    bool clean_ok = has_frame;
    for (const DevChannel& ch : hp.channels)
        for (int f = 0; f < ch.nq; ++f)
            if (hp.factors[ch.fac_off + f].antidiag) clean_ok = false;
    hp.hdr.clean_tables = clean_ok ? 1 : 0;
    if (!has_frame || clean_ok) precompute_tables(hp);
    hp.hdr.max_tab = 1;
    hp.hdr.max_stages = 1;
    for (const auto& br : hp.block_ranges) {
        hp.hdr.max_tab = std::max({hp.hdr.max_tab, br.fwd_tab, br.bwd_tab});
        hp.hdr.max_stages = std::max({hp.hdr.max_stages, br.fwd_nst, br.bwd_nst});
    }
    hp.W = S * std::max(P, 1);
    hp.W_low = S * std::max(P - 1, 0);
    return PW_OK;
}

}  // namespace pw

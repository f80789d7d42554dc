// Cache-blocking transpiler (host) -- Sec. IV.A of Doi & Horii (Listing 3) and the output
// reordering of Sec. IV.C (Fig. 10 case (b)).
//
// Readings of the points the paper leaves open (the same readings the oracle takes):
//  * QB_CHUNK holds c - reserve qubits (the listing's array bound taken as nc entries when
//    reserve = 0).
//  * Choice order: the first remaining gate's qubits (guarantees progress), then qubits of
//    multi-qubit gates in list order, then of 1-qubit gates, then already-resident qubits by
//    ascending physical bit; a gate whose new qubits do not all fit is skipped (all qubits of
//    a multi-qubit gate enter the chunk together, Sec. IV.A).
//  * A chunk_swap round pairs the incoming qubits (sorted by id) with the vacated chunk bits
//    (sorted ascending); each pair swaps physical bits (slot < c, old position >= c).
//  * Where the listing's deferral branch marks QB_CHUNK it is taken as marking QB_BLOCKED: a
//    deferred gate with any qubit in the chunk blocks all of its qubits.
//  * SWAP gates are relabels; the final reordering is a bit permutation split into two rounds
//    of disjoint transpositions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "sv_internal.h"

namespace sv {

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }

sv_plan *plan_blocking(int n, const sv_gate *gates, int64_t n_gates, const sv_options &o, SectionChooser *chooser,
                       int dtype) {
    if (n < 1 || n > 62) fail(SV_ERR_ARG, "n out of range");
    if (n_gates < 0 || (n_gates > 0 && !gates)) fail(SV_ERR_ARG, "null gate list");
    const int c = o.chunk_bits;
    if (c < 1) fail(SV_ERR_ARG, "chunk_bits must be >= 1");
    if (o.reserve != 0 && o.reserve != 1) fail(SV_ERR_ARG, "reserve must be 0 or 1");
    const int width = std::min(c, n);
    const int target = std::min(c - o.reserve, n);
    if (target < 1) fail(SV_ERR_ARG, "chunk too small");
    const int pinned = o.gather_pinned;
    if (pinned < 0 || pinned > n || (pinned && target - pinned < 2))
        fail(SV_ERR_ARG, "gather_pinned leaves no room for a 2-qubit gate");

    struct PG {
        int64_t gi;
        int32_t nq;
        int32_t lq[2];  // labels in the gate's own order
        int32_t vq[2];  // virtual qubits
        uint64_t vmask;
        bool diag;      // may join a section with qubits outside the chunk (diag_outside)
    };
    const bool diag_outside = o.diag_outside != 0 && !o.use_tc;

    auto *plan = new sv_plan();
    plan->n = n;
    plan->c = c;
    plan->reserve = o.reserve;
    plan->restore = o.restore_layout ? 1 : 0;
    // register-group width: 4 or 5 bits (3 too for tensor-core groups)
    plan->seg_bits = (o.seg_bits == 4 || o.seg_bits == 5 || (o.seg_bits == 3 && o.use_tc)) ? o.seg_bits : 4;
    plan->use_tc = o.use_tc;
    plan->pinned = pinned;
    plan->tc_no_renorm = o.tc_no_renorm ? 1 : 0;
    if (o.wait_limit_ms < 0) { delete plan; fail(SV_ERR_ARG, "wait_limit_ms must be >= 0"); }
    plan->wait_limit_ms = o.wait_limit_ms;
    plan->keys.reserve((size_t)n_gates);

    std::vector<int32_t> lab(n);
    std::iota(lab.begin(), lab.end(), 0);
    std::vector<PG> remaining;
    remaining.reserve((size_t)n_gates);
    for (int64_t i = 0; i < n_gates; ++i) {
        const sv_gate &g = gates[i];
        if (g.nq != 1 && g.nq != 2) { delete plan; fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": nq must be 1 or 2"); }
        for (int j = 0; j < g.nq; ++j)
            if (g.q[j] < 0 || g.q[j] >= n) { delete plan; fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": qubit out of range"); }
        if (g.nq == 2 && g.q[0] == g.q[1]) { delete plan; fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": repeated qubit"); }
        plan->keys.push_back(GateKey{g.nq, g.q[0], g.nq == 2 ? g.q[1] : -1, g.flags});
        if (g.flags & SV_GATE_SWAP) {
            if (g.nq != 2) { delete plan; fail(SV_ERR_ARG, "SWAP gate needs 2 qubits"); }
            std::swap(lab[g.q[0]], lab[g.q[1]]);
            continue;
        }
        if (g.nq > target) { delete plan; fail(SV_ERR_ARG, "gate " + std::to_string(i) + " is wider than the chunk"); }
        PG p{};
        p.gi = i;
        p.nq = g.nq;
        p.vmask = 0;
        p.diag = false;
        if (diag_outside && (g.flags & SV_GATE_DIAG)) {
            const int d = 1 << g.nq;
            p.diag = true;
            for (int r = 0; r < d; ++r)
                for (int cc = 0; cc < d; ++cc)
                    if (r != cc && (g.m[2 * (r * d + cc)] != 0.0 || g.m[2 * (r * d + cc) + 1] != 0.0)) p.diag = false;
        }
        for (int j = 0; j < g.nq; ++j) {
            p.lq[j] = g.q[j];
            p.vq[j] = lab[g.q[j]];
            p.vmask |= 1ull << p.vq[j];
        }
        remaining.push_back(p);
    }

    std::vector<int32_t> m(n), pinv(n);
    std::iota(m.begin(), m.end(), 0);
    std::iota(pinv.begin(), pinv.end(), 0);

    // The paper's QB_CHUNK rule for a chunk of `tgt` qubits.
    auto rule_select = [&](int tgt) {
        uint64_t chosen = 0;
        int cnt = 0;
        auto try_add = [&](uint64_t msk) {
            const uint64_t fresh = msk & ~chosen;
            if (cnt + popc(fresh) <= tgt) {
                chosen |= fresh;
                cnt += popc(fresh);
            }
        };
        for (int p = 0; p < pinned; ++p) try_add(1ull << pinv[p]);  // gathered chunks keep the low bits
        try_add(remaining.front().vmask);
        for (const PG &g : remaining) {
            if (cnt >= tgt) break;
            if (g.nq > 1) try_add(g.vmask);
        }
        for (const PG &g : remaining) {
            if (cnt >= tgt) break;
            if (g.nq == 1) try_add(g.vmask);
        }
        for (int p = 0; p < (pinned ? n : width) && cnt < tgt; ++p) try_add(1ull << pinv[p]);
        return chosen;
    };
    // Whether the QB_BLOCKED scan takes gate g into a section on `chosen` (see the scan below).
    auto takes = [&](const PG &g, uint64_t chosen, uint64_t blocked, uint64_t out_blocked) {
        const uint64_t outside = g.vmask & ~chosen;
        return outside == 0 ? (g.vmask & blocked) == 0
                            : g.diag && (g.vmask & chosen & blocked) == 0 && (outside & out_blocked) == 0;
    };
    // whether some gate may join a section with qubits outside the chunk (diag_outside)
    bool any_diag = false;
    for (const PG &g : remaining) any_diag = any_diag || g.diag;
    // The first pending gates' qubit masks, packed for the look-ahead scans (refreshed per section).
    std::vector<uint64_t> window;
    // Gates of REMAINING (at most `limit` inspected) that a section on `chosen` would take: the
    // scan in full, for plans with outside-chunk diagonals.
    auto absorbed = [&](uint64_t chosen, size_t limit) {
        uint64_t blocked = 0, out_blocked = 0;
        int k = 0;
        for (size_t i = 0; i < remaining.size() && i < limit; ++i) {
            const PG &g = remaining[i];
            if (takes(g, chosen, blocked, out_blocked)) {
                ++k;
            } else {
                if (g.vmask & chosen) blocked |= g.vmask;
                out_blocked |= g.vmask & ~chosen;
            }
        }
        return k;
    };
    // Without outside-chunk diagonals a gate is taken exactly when its qubits lie in the chunk
    // qubits not yet blocked (`open`), a gate left behind blocks the chunk qubits it touches, and
    // once every chunk qubit is blocked no later gate is taken, so the scan stops there.  The scan
    // for `chosen | fresh` runs exactly as the scan for `chosen` (with the qubits of `fresh` open
    // besides) up to the first gate that touches `fresh`, since the gates before it neither use
    // nor block those qubits.  So the scan of `chosen` is kept position by position (the count so
    // far and the open qubits before each position, frozen once it stops) and a candidate's scan
    // starts at the first use of its new qubits.
    std::vector<int> base_k;
    std::vector<uint64_t> base_open;
    int first_use[64];
    auto scan_base = [&](uint64_t chosen) {
        const size_t W = window.size();
        base_k.resize(W + 1);
        base_open.resize(W + 1);
        uint64_t open = chosen;
        int k = 0;
        size_t t = 0;
        for (; t < W; ++t) {
            base_k[t] = k;
            base_open[t] = open;
            const uint64_t v = window[t];
            const bool take = (v & ~open) == 0;
            k += take;
            open &= ~(v & (0 - (uint64_t)(!take && (v & chosen) != 0)));
            if (!open) {
                ++t;
                break;
            }
        }
        for (; t <= W; ++t) {
            base_k[t] = k;
            base_open[t] = open;
        }
    };
    auto absorbed_with = [&](uint64_t chosen, uint64_t fresh) {
        const size_t W = window.size();
        size_t t0 = W;
        for (uint64_t f = fresh; f; f &= f - 1) t0 = std::min(t0, (size_t)first_use[__builtin_ctzll(f)]);
        const uint64_t ch = chosen | fresh;
        uint64_t open = base_open[t0] | fresh;
        int k = base_k[t0];
        for (size_t i = t0; i < W; ++i) {  // the scan above, without data-dependent branches
            const uint64_t v = window[i];
            const bool take = (v & ~open) == 0;
            k += take;
            open &= ~(v & (0 - (uint64_t)(!take && (v & ch) != 0)));
            if (!open) break;
        }
        return k;
    };
    // Look-ahead alternative (cost-model candidates only): grow the chunk from the pinned bits
    // and the first gate by the pending gate whose qubits add the most absorbable gates.
    auto greedy_select = [&](int tgt) {
        constexpr size_t kWindow = 512, kChoices = 64;
        window.clear();
        for (size_t i = 0; i < remaining.size() && i < kWindow; ++i) window.push_back(remaining[i].vmask);
        for (int b = 0; b < 64; ++b) first_use[b] = (int)window.size();
        for (size_t i = window.size(); i-- > 0;)
            for (uint64_t v = window[i]; v; v &= v - 1) first_use[__builtin_ctzll(v)] = (int)i;
        uint64_t chosen = remaining.front().vmask;
        for (int p = 0; p < pinned; ++p) chosen |= 1ull << pinv[p];
        uint64_t seen[64];  // the new-qubit sets tried, one bit per pair (lower qubit, higher qubit)
        while (popc(chosen) < tgt) {
            uint64_t best = 0;
            int best_score = -1;
            size_t tried = 0;
            std::memset(seen, 0, sizeof(seen));
            if (!any_diag) scan_base(chosen);
            const int room = tgt - popc(chosen);
            for (size_t i = 0; i < window.size() && tried < kChoices; ++i) {
                const uint64_t fresh = window[i] & ~chosen;
                if (!fresh) continue;
                // a gate has at most two qubits
                const uint64_t rest = fresh & (fresh - 1);
                if ((rest ? 2 : 1) > room) continue;
                const int lo = __builtin_ctzll(fresh), hi = rest ? __builtin_ctzll(rest) : lo;
                if ((seen[lo] >> hi) & 1) continue;
                seen[lo] |= 1ull << hi;
                ++tried;
                const int sc = any_diag ? absorbed(chosen | fresh, kWindow) : absorbed_with(chosen, fresh);
                if (sc > best_score) {
                    best_score = sc;
                    best = fresh;
                }
            }
            if (!best) break;
            chosen |= best;
        }
        for (int p = 0; p < n && popc(chosen) < tgt; ++p) chosen |= 1ull << pinv[p];
        return chosen;
    };

    std::vector<PG> next;
    std::vector<SectionCandidate> cands;
    while (!remaining.empty()) {
        // choose QB_CHUNK
        uint64_t chosen = (pinned && o.lookahead && !chooser) ? greedy_select(target) : rule_select(target);
        int chosen_r = 0;  // this section's register-group width (0: the plan's)
        if (chooser && pinned) {
            cands.clear();
            auto make_candidate = [&](uint64_t ch, int r) {
                SectionCandidate cd;
                cd.chosen = ch;
                cd.ce = popc(ch);
                cd.seg_bits = r;
                PlanOp tmp;
                tmp.kind = 4;
                tmp.seg_bits = r;
                uint64_t blocked = 0, out_blocked = 0;
                for (const PG &g : remaining) {
                    if (takes(g, ch, blocked, out_blocked)) {
                        BlockGate bg{};
                        bg.gi = g.gi;
                        bg.nq = g.nq;
                        for (int j = 0; j < g.nq; ++j) bg.phys[j] = m[g.vq[j]];
                        if (g.nq == 1) bg.phys[1] = -1;
                        tmp.gates.push_back(bg);
                    } else {
                        if (g.vmask & ch) blocked |= g.vmask;
                        out_blocked |= g.vmask & ~ch;
                    }
                }
                for (int v = 0; v < n; ++v)
                    if ((ch >> v) & 1) tmp.mask |= 1ull << m[v];
                cd.absorbed = (int)tmp.gates.size();
                section_features(*plan, tmp, gates, dtype, cd.f);
                return cd;
            };
            auto add_candidate = [&](uint64_t ch) {
                for (const SectionCandidate &c0 : cands)
                    if (c0.chosen == ch) return;
                cands.push_back(make_candidate(ch, 0));
            };
            add_candidate(chosen);
            // smaller chunks (still room for a 2-qubit gate; >= 11 bits for the tensor-core path)
            const int min_t = std::max(pinned + 2, (o.use_tc && dtype == SV_C64) ? plan->seg_bits + 7 : 1);
            for (int d = 1; d <= 2; ++d)
                if (target - d >= min_t && target - d >= remaining.front().nq + pinned) add_candidate(rule_select(target - d));
            add_candidate(greedy_select(target));
            chosen = cands[(size_t)std::max(0, std::min((int)cands.size() - 1, chooser->choose(cands)))].chosen;
            // the register-group width of the section's tensor-core groups: the plan's, or 4 or 5
            // bits where the chunk has room (at least 2^(r+7) amplitudes), as the chooser picks
            // (every width takes the same gates, so the model's choice is the lowest predicted time)
            if (o.use_tc && dtype == SV_C64) {
                std::vector<SectionCandidate> widths;
                const int ce = popc(chosen);
                for (int r : {plan->seg_bits, 4, 5}) {
                    bool dup = false;
                    for (const SectionCandidate &w0 : widths) dup = dup || w0.seg_bits == r;
                    if (!dup && ce >= r + 7) widths.push_back(make_candidate(chosen, r));
                }
                if (widths.size() > 1)
                    chosen_r = widths[(size_t)std::max(0, std::min((int)widths.size() - 1, chooser->choose(widths)))].seg_bits;
            }
        }

        // chunk_swap round (none for gathered chunks: the section fetches its bits in place)
        PlanOp round;
        round.kind = 1;
        std::vector<int32_t> incoming, vacated;
        for (int v = 0; v < n && !pinned; ++v)
            if (((chosen >> v) & 1) && m[v] >= width) incoming.push_back(v);
        for (int p = 0; p < width; ++p)
            if (!((chosen >> pinv[p]) & 1)) vacated.push_back(p);
        for (size_t k = 0; k < incoming.size(); ++k) {
            const int v_in = incoming[k], slot = vacated[k];
            const int old = m[v_in], v_out = pinv[slot];
            m[v_in] = slot;
            pinv[slot] = v_in;
            m[v_out] = old;
            pinv[old] = v_out;
            round.pairs.emplace_back(slot, old);
        }
        if (!round.pairs.empty()) plan->ops.push_back(std::move(round));

        // scan REMAINING with QB_BLOCKED
        PlanOp block;
        block.kind = pinned ? 4 : 2;
        block.seg_bits = chosen_r == plan->seg_bits ? 0 : chosen_r;
        if (pinned)
            for (int v = 0; v < n; ++v)
                if ((chosen >> v) & 1) block.mask |= 1ull << m[v];
        // diag_outside: a diagonal gate may also take qubits outside the chunk (constant over a
        // chunk), provided no earlier deferred gate touches those qubits (OUT_BLOCKED), so the
        // per-qubit gate order is kept
        uint64_t blocked = 0, out_blocked = 0;
        next.clear();
        for (const PG &g : remaining) {
            const uint64_t outside = g.vmask & ~chosen;
            if (takes(g, chosen, blocked, out_blocked)) {
                BlockGate bg{};
                bg.gi = g.gi;
                bg.nq = g.nq;
                for (int j = 0; j < g.nq; ++j) {
                    bg.phys[j] = m[g.vq[j]];
                    bg.label[j] = g.lq[j];
                }
                if (g.nq == 1) { bg.phys[1] = -1; bg.label[1] = -1; }
                block.gates.push_back(bg);
            } else {
                next.push_back(g);
                if (g.vmask & chosen) blocked |= g.vmask;
                out_blocked |= outside;
            }
        }
        plan->ops.push_back(std::move(block));
        remaining.swap(next);
    }

    // output reordering: bit src[q] = m[lab[q]] must move to bit q
    std::vector<int32_t> src(n);
    for (int q = 0; q < n; ++q) src[q] = m[lab[q]];
    if (plan->restore) {
        std::vector<int32_t> dest(n);
        for (int q = 0; q < n; ++q) dest[src[q]] = q;
        PlanOp r1, r2;
        r1.kind = r2.kind = 3;
        std::vector<char> seen(n, 0);
        for (int x0 = 0; x0 < n; ++x0) {
            if (seen[x0]) continue;
            std::vector<int32_t> cyc{x0};
            seen[x0] = 1;
            for (int y = dest[x0]; y != x0; y = dest[y]) {
                cyc.push_back(y);
                seen[y] = 1;
            }
            const int L = (int)cyc.size();
            if (L == 1) continue;
            for (int i = 1; i <= (L - 1) / 2; ++i) {
                int a = cyc[i], b = cyc[L - i];
                r1.pairs.emplace_back(std::min(a, b), std::max(a, b));
            }
            for (int i = 1; i <= L / 2; ++i) {
                int a = cyc[i], b = cyc[(L + 1 - i) % L];
                r2.pairs.emplace_back(std::min(a, b), std::max(a, b));
            }
        }
        for (PlanOp *r : {&r1, &r2}) {
            if (r->pairs.empty()) continue;
            std::sort(r->pairs.begin(), r->pairs.end());
            plan->ops.push_back(std::move(*r));
        }
        plan->final_map.resize(n);
        std::iota(plan->final_map.begin(), plan->final_map.end(), 0);
    } else {
        plan->final_map = src;
    }

    return plan;
}

// ---------------------------------------------------------------------------------------
// Register groups.  Inside a blocking section each chunk lives in shared memory; a group is
// a set of r chunk bits whose 2^r amplitudes one thread holds in registers while it applies
// every gate of the group.  A group on bits S takes, in section order, every pending gate inside
// S, and a gate that is not taken blocks its bits for the rest of the group (so per-qubit gate
// order is kept) -- the transpiler's QB_BLOCKED rule one level down.  Each group costs the
// section one pass over its chunk, so the groups are chosen to be few: a beam search over the
// pending gate lists (beam_groups below); a group is an r-subset of the bits the pending gates
// use (a superset of bits takes a superset of the gates, so r-subsets suffice).  A section whose
// search exceeds its budget falls back to the greedy choice: the first pending gate's bits,
// grown one pending gate at a time (the first 64 with new bits) by the one that lets the group
// take the most gates.
//
// Lane layout: the lanes that share a shared-memory wavefront (16 for 8-byte amplitudes, 8 for
// 16-byte ones) must enumerate distinct bank slots.  A chunk bit k contributes the slot vector
// w(k) = 2^k for k < SB and the swizzle pattern V[k] above; the first lane bits are chosen
// greedily (ascending bit order) among the bits outside the group so that their w(k) are
// linearly independent over GF(2).
namespace {

// Gates of `pending` a group on `bits` takes (in order) and the rest.
void split_pending(const std::vector<uint64_t> &mask, const std::vector<int32_t> &pending, uint64_t bits,
                   std::vector<int32_t> *taken, std::vector<int32_t> &rest) {
    uint64_t blocked = 0;
    rest.clear();
    for (int32_t idx : pending) {
        const uint64_t mk = mask[idx];
        if ((mk & ~bits) == 0 && (mk & blocked) == 0) {
            if (taken) taken->push_back(idx);
        } else {
            blocked |= mk;
            rest.push_back(idx);
        }
    }
}

// Groups by beam search: level by level, every r-subset of the bits the pending gates use is
// tried on each of the `width` pending lists kept (subsets in lexicographic order of their bit
// positions); the children are ranked by the lower bound ceil(|bits used| / r) on the groups they
// still need, then by pending gates, then by bits used (stable: ties keep the order they were
// found in), and the first list to empty ends the search.  Returns false once the budget is spent
// (each subset tried counts the length of the pending list it is tried on).
constexpr int kGroupBeam = 8;
constexpr int kGroupBeamMaxGates = 32;  // sections with more gates search with a beam of one
constexpr int64_t kGroupSearchBudget = 4000000;  // per section: pending-list length summed over the subsets tried

bool beam_groups(const std::vector<uint64_t> &mask, int r, std::vector<uint64_t> &out, int width) {
    const int G = (int)mask.size();
    if (G == 0) return true;
    bool any_zero = false;  // a gate with no chunk bit fits every group, so no scan may stop early
    for (uint64_t mk : mask) any_zero = any_zero || mk == 0;
    // the groups chosen so far, as a tree: each kept list points at its parent's entry
    struct Chosen {
        uint64_t set;
        int parent;
    };
    std::vector<Chosen> tree;
    auto finish = [&](int at, uint64_t last) {
        out.clear();
        for (int i = at; i >= 0; i = tree[(size_t)i].parent) out.push_back(tree[(size_t)i].set);
        std::reverse(out.begin(), out.end());
        out.push_back(last);
        return true;
    };
    struct Node {
        std::vector<int32_t> pend;
        int at;  // its last group in `tree`, -1 for none
    };
    // A level's children in rank order (lower bound, pending gates, bits used, then the order they
    // were found in).  Only the best `width` distinct lists survive a level, so at most `width` are
    // kept while the level runs: a later duplicate of a list ties with it and comes after it, so it
    // can neither displace it nor enter once it has been pushed out.  A child's pending list is
    // written out only when it enters.
    struct Child {
        std::vector<int32_t> pend;
        uint64_t set;
        int parent, lb, npend, nbits;
        int64_t order;
    };
    auto better = [](const Child &a, const Child &b) {
        if (a.lb != b.lb) return a.lb < b.lb;
        if (a.npend != b.npend) return a.npend < b.npend;
        if (a.nbits != b.nbits) return a.nbits < b.nbits;
        return a.order < b.order;
    };
    std::vector<Node> beam(1);
    beam[0].pend.resize((size_t)G);
    std::iota(beam[0].pend.begin(), beam[0].pend.end(), 0);
    beam[0].at = -1;
    std::vector<Child> top;
    std::vector<uint64_t> suffix;  // suffix[j]: the bits of pend[j..]
    int64_t budget = kGroupSearchBudget;
    while (true) {
        top.clear();
        int64_t found = 0;
        for (const Node &nd : beam) {
            const std::vector<int32_t> &pend = nd.pend;
            const int P = (int)pend.size();
            suffix.assign((size_t)P + 1, 0);
            for (int j = P - 1; j >= 0; --j) suffix[(size_t)j] = suffix[(size_t)j + 1] | mask[(size_t)pend[(size_t)j]];
            const uint64_t used = suffix[0];
            if (popc(used) <= r) return finish(nd.at, used);  // one more group takes every pending gate
            int bits[64], nb = 0;
            for (int b = 0; b < 64; ++b)
                if ((used >> b) & 1) bits[nb++] = b;
            int sel[8];
            for (int k = 0; k < r; ++k) sel[k] = k;
            while (true) {
                budget -= P;
                if (budget < 0) return false;
                uint64_t set = 0;
                for (int k = 0; k < r; ++k) set |= 1ull << bits[sel[k]];
                // the gates the group takes, and the bits of those it leaves (once every bit of the
                // group is blocked nothing later fits, and the rest of the list is left as it is)
                uint64_t blocked = 0, left = 0;
                int taken = 0, stop = P;
                for (int j = 0; j < P; ++j) {
                    const uint64_t mk = mask[(size_t)pend[(size_t)j]];
                    if ((mk & ~set) == 0 && (mk & blocked) == 0) {
                        ++taken;
                    } else {
                        blocked |= mk;
                        left |= mk;
                        if (!any_zero && (blocked & set) == set) {
                            stop = j + 1;
                            break;
                        }
                    }
                }
                if (taken == P) return finish(nd.at, set);
                if (taken > 0) {
                    Child ch;
                    ch.set = set;
                    ch.parent = nd.at;
                    ch.nbits = popc(left | suffix[(size_t)stop]);
                    ch.lb = (ch.nbits + r - 1) / r;
                    ch.npend = P - taken;
                    ch.order = found++;
                    if ((int)top.size() < width || better(ch, top.back())) {
                        ch.pend.reserve((size_t)ch.npend);
                        blocked = 0;
                        for (int j = 0; j < stop; ++j) {
                            const uint64_t mk = mask[(size_t)pend[(size_t)j]];
                            if ((mk & ~set) != 0 || (mk & blocked) != 0) {
                                blocked |= mk;
                                ch.pend.push_back(pend[(size_t)j]);
                            }
                        }
                        ch.pend.insert(ch.pend.end(), pend.begin() + stop, pend.end());
                        bool dup = false;
                        for (const Child &t : top) dup = dup || t.pend == ch.pend;
                        if (!dup) {
                            size_t at = top.size();
                            while (at > 0 && better(ch, top[at - 1])) --at;
                            top.insert(top.begin() + (std::ptrdiff_t)at, std::move(ch));
                            if ((int)top.size() > width) top.pop_back();
                        }
                    }
                }
                // next r-subset of [0, nb) in lexicographic order
                int k = r - 1;
                while (k >= 0 && sel[k] == nb - r + k) --k;
                if (k < 0) break;
                ++sel[k];
                for (int q = k + 1; q < r; ++q) sel[q] = sel[q - 1] + 1;
            }
        }
        beam.clear();
        for (Child &c : top) {
            tree.push_back(Chosen{c.set, c.parent});
            beam.push_back(Node{std::move(c.pend), (int)tree.size() - 1});
        }
    }
}

}  // namespace

std::vector<HostSeg> segment_block(const std::vector<BlockGate> &gates, int width, int r, int elem_bytes, bool search) {
    std::vector<HostSeg> segs;
    std::vector<int32_t> pending(gates.size());
    std::iota(pending.begin(), pending.end(), 0);
    std::vector<uint64_t> mask(gates.size());  // chunk bits only (a qubit outside has phys -1)
    for (size_t i = 0; i < gates.size(); ++i) {
        uint64_t mk = 0;
        for (int j = 0; j < gates[i].nq; ++j)
            if (gates[i].phys[j] >= 0) mk |= 1ull << gates[i].phys[j];
        mask[i] = mk;
    }
    const int rr = std::min(r, width);
    // the group sets: the search's, else the greedy choice
    std::vector<uint64_t> sets;
    // long sections (whole small-state circuits in one residency) search with a beam of one: the
    // full beam's cost grows with the pending lists, and its gain there is a few per cent
    const int beam = (int)gates.size() > kGroupBeamMaxGates ? 1 : kGroupBeam;
    if (!search || !beam_groups(mask, rr, sets, beam)) sets.clear();
    if (sets.empty() && !pending.empty()) {
        // a gate with no chunk bit (a diagonal wholly outside the chunk) fits every group
        bool any_outside = false;
        for (uint64_t mk : mask) any_outside = any_outside || mk == 0;
        std::vector<int32_t> pend = pending, rest;
        // gates a group on `bits` takes: in order, those inside `bits` and not behind a deferred
        // gate (once all of `bits` are blocked no later gate fits, unless it has no chunk bit)
        auto takes = [&](uint64_t bits) {
            uint64_t blocked = 0;
            int k = 0;
            for (int32_t idx : pend) {
                const uint64_t mk = mask[idx];
                if ((mk & ~bits) == 0 && (mk & blocked) == 0) {
                    ++k;
                } else {
                    blocked |= mk;
                    if (!any_outside && (blocked & bits) == bits) break;
                }
            }
            return k;
        };
        while (!pend.empty()) {
            uint64_t set = mask[pend.front()];
            while (popc(set) < rr) {
                uint64_t best = 0;
                int best_k = -1;
                size_t tried = 0;
                for (size_t i = 0; i < pend.size() && tried < 64; ++i) {
                    const uint64_t fresh = mask[pend[i]] & ~set;
                    if (!fresh || popc(set | fresh) > rr) continue;
                    ++tried;
                    const int k = takes(set | fresh);
                    if (k > best_k) {
                        best_k = k;
                        best = fresh;
                    }
                }
                if (!best) break;
                set |= best;
            }
            sets.push_back(set);
            split_pending(mask, pend, set, nullptr, rest);
            pend.swap(rest);
        }
    }
    std::vector<int32_t> rest;
    for (uint64_t set : sets) {
        HostSeg s;
        s.r = rr;
        split_pending(mask, pending, set, &s.gates, rest);
        // pad with the highest unused chunk bits (keeps the low bits free for the lanes)
        for (int p = width - 1; p >= 0 && popc(set) < rr; --p)
            if (!((set >> p) & 1)) set |= 1ull << p;
        int k = 0;
        for (int p = 0; p < width && k < rr; ++p)
            if ((set >> p) & 1) s.pos[k++] = p;
        segs.push_back(std::move(s));
        pending.swap(rest);
    }
    // lane layouts
    const int sb = elem_bytes == 8 ? 4 : 3;
    const int *swz = elem_bytes == 8 ? kSwz64 : kSwz128;
    for (size_t i = 0; i < segs.size(); ++i) {
        HostSeg &s = segs[i];
        uint64_t in = 0;
        for (int k = 0; k < s.r; ++k) in |= 1ull << s.pos[k];
        std::vector<int> outside;
        for (int p = 0; p < width; ++p)
            if (!((in >> p) & 1)) outside.push_back(p);
        std::vector<int> lanes, others;
        int basis[8] = {0};  // GF(2) echelon basis by leading bit
        for (int p : outside) {
            if ((int)lanes.size() < sb) {
                int v = p < sb ? (1 << p) : swz[p];
                for (int b = sb - 1; b >= 0 && v; --b)
                    if ((v >> b) & 1) {
                        if (basis[b]) v ^= basis[b];
                        else { basis[b] = v; v = -1; break; }
                    }
                if (v == -1) { lanes.push_back(p); continue; }
            }
            others.push_back(p);
        }
        // complete the lane bits (5 in all) from the remaining bits, lowest first
        std::vector<int> order = lanes;
        std::vector<int> rem;
        for (int p : others) {
            if ((int)order.size() < 5) order.push_back(p);
            else rem.push_back(p);
        }
        // if fewer than sb independent bits existed, the first lanes are whatever is available
        for (int j = 0; j < 5; ++j) s.lane[j] = j < (int)order.size() ? order[j] : 0;
        s.nrest = (int)rem.size();
        for (int j = 0; j < s.nrest; ++j) s.rest[j] = rem[j];
        s.flags = (i == 0 ? 1 : 0) | (i + 1 == segs.size() ? 2 : 0);
    }
    return segs;
}

// Gathered chunk layout: runs of consecutive chunk bits; the run at bit 0 and the (up to) four
// longest other runs start tensor dimensions (boxes of at most 8 bits, 7 for the doubled
// complex128 innermost dimension), everything else in the chunk is a loop bit.
GatherLayout gather_layout(uint64_t mask, int n, int elem_bytes) {
    GatherLayout L;
    for (int b = 0; b < 64; ++b) L.local_of[b] = -1;
    std::vector<std::pair<int, int>> runs;  // (start, length)
    for (int b = 0; b < n;) {
        if ((mask >> b) & 1) {
            const int s = b;
            while (b < n && ((mask >> b) & 1)) ++b;
            runs.emplace_back(s, b - s);
        } else {
            ++b;
        }
    }
    if (runs.empty() || runs[0].first != 0) fail(SV_ERR_PLAN, "a gathered chunk must contain bit 0");
    std::vector<int> idx;
    for (int i = 1; i < (int)runs.size(); ++i) idx.push_back(i);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return runs[a].second > runs[b].second; });
    if (idx.size() > 4) idx.resize(4);
    std::sort(idx.begin(), idx.end());
    std::vector<int> dims{0};
    dims.insert(dims.end(), idx.begin(), idx.end());
    GatherArgs &A = L.args;
    A.rank = (int)dims.size();
    int k = 0, box_bits = 0;
    for (int d = 0; d < A.rank; ++d) {
        A.s[d] = runs[dims[d]].first;
        const int cap = d == 0 ? (elem_bytes == 8 ? 8 : 7) : 8;
        L.box_len[d] = std::min(runs[dims[d]].second, cap);
        for (int b = A.s[d]; b < A.s[d] + L.box_len[d]; ++b) L.local_of[b] = k++;
        box_bits += L.box_len[d];
    }
    A.s[A.rank] = n;
    A.nloop = 0;
    A.nouter = 0;
    for (int b = 0; b < n; ++b) {
        if ((mask >> b) & 1) {
            if (L.local_of[b] < 0) {
                if (A.nloop >= 16) fail(SV_ERR_UNSUPPORTED, "gathered chunk has too many scattered bits");
                A.loop[A.nloop++] = (int8_t)b;
                L.local_of[b] = k++;
            }
        } else {
            A.outer[A.nouter++] = (int8_t)b;
        }
    }
    A.box_amps = 1 << box_bits;
    L.ce = k;
    return L;
}

std::vector<BlockGate> localize_gates(const PlanOp &op, int n, int c, const GatherLayout *lay) {
    const int width = std::min(c, n);
    std::vector<BlockGate> loc = op.gates;
    for (BlockGate &g : loc) {
        for (int j = 0; j < g.nq; ++j) {
            const int p = g.phys[j];
            const int l = lay ? lay->local_of[p] : (p < width ? p : -1);
            g.ext[j] = l < 0 ? p : -1;
            g.phys[j] = l;
        }
    }
    return loc;
}

template <typename T>
void encode_gate(const sv_gate &g, const BlockGate &bg, const HostSeg &seg, DevGate<T> &out) {
    auto local = [&](int phys) {
        for (int k = 0; k < seg.r; ++k)
            if (seg.pos[k] == phys) return k;
        fail(SV_ERR_PLAN, "gate bit outside its register group");
    };
    std::memset(&out, 0, sizeof(out));
    if (bg.ext[0] >= 0 || (g.nq == 2 && bg.ext[1] >= 0)) {
        // diagonal gate with qubits outside the chunk: per value of the outside bits, the
        // diagonal it leaves on its chunk qubit (or the phase it applies)
        const int d = 1 << g.nq;
        double D[8];
        for (int i = 0; i < d; ++i) {
            D[2 * i] = g.m[2 * (i * d + i)];
            D[2 * i + 1] = g.m[2 * (i * d + i) + 1];
        }
        out.op = OP_DIAGX;
        auto put = [&](int v, int i_lo, int i_hi) {
            out.m[4 * v] = (T)D[2 * i_lo];
            out.m[4 * v + 1] = (T)D[2 * i_lo + 1];
            out.m[4 * v + 2] = (T)D[2 * i_hi];
            out.m[4 * v + 3] = (T)D[2 * i_hi + 1];
        };
        int e0 = 0xFF, e1 = 0xFF;
        // a phase is written as the diagonal (d, d) on register bit 0
        if (g.nq == 1) {  // phase d[x], x = the qubit's bit
            out.a = 0;
            e0 = bg.ext[0];
            put(0, 0, 0);
            put(1, 1, 1);
        } else if (bg.ext[0] >= 0 && bg.ext[1] >= 0) {  // phase d[x0 + 2 x1]
            out.a = 0;
            e0 = bg.ext[0];
            e1 = bg.ext[1];
            for (int v = 0; v < 4; ++v) put(v, v, v);
        } else if (bg.ext[1] >= 0) {  // q0 in the chunk: diag(d[2x], d[1 + 2x]) on it
            out.a = local(bg.phys[0]);
            e0 = bg.ext[1];
            put(0, 0, 1);
            put(1, 2, 3);
        } else {  // q1 in the chunk: diag(d[x], d[x + 2]) on it
            out.a = local(bg.phys[1]);
            e0 = bg.ext[0];
            put(0, 0, 2);
            put(1, 1, 3);
        }
        out.b = e0 | (e1 << 8);
        out.code = out.a;
        return;
    }
    if (g.nq == 1) {
        out.a = local(bg.phys[0]);
        out.b = -1;
        out.code = out.a;
        const bool diag = g.m[2] == 0.0 && g.m[3] == 0.0 && g.m[4] == 0.0 && g.m[5] == 0.0;
        if (diag) {
            out.op = OP_DIAG1;
            out.m[0] = (T)g.m[0]; out.m[1] = (T)g.m[1];
            out.m[2] = (T)g.m[6]; out.m[3] = (T)g.m[7];
        } else {
            static const double kX[8] = {0, 0, 1, 0, 1, 0, 0, 0};
            bool flip = true;
            for (int i = 0; i < 8; ++i) flip = flip && g.m[i] == kX[i];
            out.op = flip ? OP_X1 : OP_DENSE1;
            for (int i = 0; i < 8; ++i) out.m[i] = (T)g.m[i];
        }
        return;
    }
    int la = local(bg.phys[0]), lb = local(bg.phys[1]);
    // matrix in local basis bit(la) + 2*bit(lb); reorder so that the lower register bit is
    // the low local bit.
    double mm[32];
    if (la < lb) {
        std::memcpy(mm, g.m, sizeof(mm));
    } else {
        auto sw = [](int i) { return ((i & 1) << 1) | ((i >> 1) & 1); };
        for (int r = 0; r < 4; ++r)
            for (int cc = 0; cc < 4; ++cc) {
                mm[2 * (r * 4 + cc)] = g.m[2 * (sw(r) * 4 + sw(cc))];
                mm[2 * (r * 4 + cc) + 1] = g.m[2 * (sw(r) * 4 + sw(cc)) + 1];
            }
        std::swap(la, lb);
    }
    out.a = la;
    out.b = lb;
    out.code = la * 8 + lb;
    bool diag = true, perm = true;
    for (int r = 0; r < 4; ++r) {
        int ones = 0;
        for (int cc = 0; cc < 4; ++cc) {
            const double re = mm[2 * (r * 4 + cc)], im = mm[2 * (r * 4 + cc) + 1];
            if (r != cc && (re != 0.0 || im != 0.0)) diag = false;
            if (re == 1.0 && im == 0.0) ++ones;
            else if (re != 0.0 || im != 0.0) perm = false;
        }
        if (ones != 1) perm = false;
    }
    if (diag) {
        out.op = OP_DIAG2;
        for (int r = 0; r < 4; ++r) {
            out.m[2 * r] = (T)mm[2 * (r * 4 + r)];
            out.m[2 * r + 1] = (T)mm[2 * (r * 4 + r) + 1];
        }
    } else if (perm) {
        // m[r] = source column of output row r
        int pm[4] = {0, 0, 0, 0};
        for (int r = 0; r < 4; ++r)
            for (int cc = 0; cc < 4; ++cc)
                if (mm[2 * (r * 4 + cc)] == 1.0) pm[r] = cc;
        for (int r = 0; r < 4; ++r) out.m[r] = (T)pm[r];
        auto is = [&](int a0, int a1, int a2, int a3) { return pm[0] == a0 && pm[1] == a1 && pm[2] == a2 && pm[3] == a3; };
        out.op = is(0, 3, 2, 1) ? OP_CXA : is(0, 1, 3, 2) ? OP_CXB : is(0, 2, 1, 3) ? OP_SWAP2 : OP_PERM2;
    } else {
        out.op = OP_DENSE2;
        for (int i = 0; i < 32; ++i) out.m[i] = (T)mm[i];
    }
}

// Register groups over all blocking sections of a plan (statistics; the same groups the section
// programs get).
int plan_segment_count(const sv_plan &plan) {
    int nseg = 0;
    const int n = plan.n, c = plan.c;
    for (const PlanOp &op : plan.ops) {
        // tensor-core plans: the section's width; SIMT register groups have 4 or 5 bits
        const int r = plan.use_tc ? (op.seg_bits ? op.seg_bits : plan.seg_bits) : (plan.seg_bits == 5 ? 5 : 4);
        if (op.kind == 2)
            nseg += (int)segment_block(localize_gates(op, n, c, nullptr), std::min(c, n), r, 8).size();
        if (op.kind == 4) {
            const GatherLayout L = gather_layout(op.mask, n, 8);
            nseg += (int)segment_block(localize_gates(op, n, c, &L), L.ce, r, 8).size();
        }
    }
    return nseg;
}

// A gate that costs no multiplication-heavy work: diagonal, or a permutation (entries 0 / 1).
static bool gate_is_cheap(const sv_gate &g) {
    const int d = 1 << g.nq;
    bool diag = true, perm = true;
    for (int r = 0; r < d; ++r) {
        int ones = 0;
        for (int c = 0; c < d; ++c) {
            const double re = g.m[2 * (r * d + c)], im = g.m[2 * (r * d + c) + 1];
            const bool zero = re == 0.0 && im == 0.0;
            if (r != c && !zero) diag = false;
            if (re == 1.0 && im == 0.0) ++ones;
            else if (!zero) perm = false;
        }
        if (ones != 1) perm = false;
    }
    return diag || perm;
}

// Features of one blocking section for the cost model (all roughly in [0, 1]):
//  0 chunk bits / 16          1 register-group width / 8     2 log2(1 + gates) / 10
//  3 log2(1 + groups) / 6     4..9 share of gate-qubit chunk positions in bins {0},{1},{2},{3},
//  {4..7},{8..}               10 share of 2-qubit gates       11 share of diagonal/permutation gates
//  12 complex128              13 n / 32                       14 tensor-core sweeps / 4 (0 = SIMT)
//  15 gathered chunk
void section_features(const sv_plan &plan, const PlanOp &op, const sv_gate *gates, int dtype, float *out) {
    for (int k = 0; k < kNumFeatures; ++k) out[k] = 0.f;
    const int n = plan.n;
    std::vector<BlockGate> loc;
    int ce = std::min(plan.c, n);
    if (op.kind == 4) {
        const GatherLayout L = gather_layout(op.mask, n, 8);
        loc = localize_gates(op, n, plan.c, &L);
        ce = L.ce;
    } else {
        loc = localize_gates(op, n, plan.c, nullptr);
    }
    const int tc_r = op.seg_bits ? op.seg_bits : plan.seg_bits;
    const bool tc = plan.use_tc && dtype == SV_C64 && ce >= tc_r + 7;
    const int r = tc ? tc_r : (dtype == SV_C64 && plan.seg_bits == 5 ? 5 : 4);
    const int nseg = loc.empty() ? 0 : (int)segment_block(loc, ce, r, 8).size();
    int q_total = 0, two = 0, cheap = 0;
    float hist[6] = {0, 0, 0, 0, 0, 0};
    for (const BlockGate &g : loc) {
        two += g.nq == 2;
        cheap += gate_is_cheap(gates[g.gi]);
        for (int j = 0; j < g.nq; ++j) {
            const int p = g.phys[j];
            if (p < 0) continue;  // outside the chunk
            hist[p < 4 ? p : (p < 8 ? 4 : 5)] += 1.f;
            ++q_total;
        }
    }
    const float ng = (float)loc.size();
    out[0] = ce / 16.f;
    out[1] = r / 8.f;
    out[2] = std::log2(1.f + ng) / 10.f;
    out[3] = std::log2(1.f + (float)nseg) / 6.f;
    for (int b = 0; b < 6; ++b) out[4 + b] = q_total ? hist[b] / (float)q_total : 0.f;
    out[10] = ng > 0 ? two / ng : 0.f;
    out[11] = ng > 0 ? cheap / ng : 0.f;
    out[12] = dtype == SV_C128 ? 1.f : 0.f;
    out[13] = n / 32.f;
    out[14] = tc ? (float)((nseg + 10) / 11) / 4.f : 0.f;
    out[15] = op.kind == 4 ? 1.f : 0.f;
}

template void encode_gate<float>(const sv_gate &, const BlockGate &, const HostSeg &, DevGate<float> &);
template void encode_gate<double>(const sv_gate &, const BlockGate &, const HostSeg &, DevGate<double> &);

}  // namespace sv

"""Cache-blocking transpiler, oracle side (test infrastructure only).

Restates Sec. IV.A (Listing 3) of Doi & Horii step by step in the paper's names, with the
readings below for the points the paper leaves silent or garbled.  The CUDA library has its
own C++ implementation; the two must produce the same schedule bit for bit.

Algorithm (logical qubit -> physical bit map ``m``, inverse ``pinv``):

  REMAINING <- gate sequence (SWAP gates removed as relabels, see below)
  while REMAINING is not empty:                       # stop condition taken as: REMAINING empty
    choose QB_CHUNK: c - reserve logical qubits       # the array bound taken as nc entries, reserve = 0
        priority: (1) qubits of the first remaining gate, (2) qubits of multi-qubit gates in
        list order, (3) qubits of 1-qubit gates in list order, (4) qubits already resident
        (physical < c) by ascending physical bit; a gate whose new qubits do not all fit is
        skipped (Sec. IV.A requires every qubit of a multi-qubit gate to be in the chunk
        together).
    put chunk_swap gates in OUTPUT                    # one swap round
        incoming chosen qubits (physical >= c) sorted by logical id are paired with vacated
        physical bits (< c, held by unchosen qubits) sorted ascending; each pair is
        chunk_swap(slot, old_position) (Sec. IV.C, Fig. 10 case (a)).
    clear QB_BLOCKED
    for gate in REMAINING:
      if all its qubits in QB_CHUNK and none in QB_BLOCKED: put gate in OUTPUT (block)
      else: put gate in REMAINING_NEXT; if some of its qubits are in QB_CHUNK, set all of its
            qubits in QB_BLOCKED            # the listing marks QB_CHUNK here; taken as QB_BLOCKED
    REMAINING <- REMAINING_NEXT

SWAP gates are relabels: a SWAP(a, b) in the input exchanges which virtual qubit carries labels
a and b; later gates are rewritten, no data moves.  At the end the output is reordered so that
physical bit q holds logical qubit q (Sec. IV.C: the qubits are put back in order for the output, Fig. 10 case
(b)).  That reordering is a bit permutation, written as two rounds of disjoint transpositions:
for each cycle x0 -> x1 -> ... (x0 its smallest bit, x_{i+1} = destination of x_i) the first
round exchanges x_i <-> x_{L-i} and the second x_i <-> x_{L+1-i} (indices mod L).

Diagonal gates (``diag_outside``): a gate whose matrix is diagonal (Z, RZ, CP, CZ) may join a
section while some of its qubits are outside the chunk, because those qubits are constant over a
chunk -- the gate acts there as a diagonal on its chunk qubits, or as a phase.  It is taken when
its chunk qubits are not in QB_BLOCKED and no earlier deferred gate touches its outside qubits.

Look-ahead chunk choice (``lookahead``, gathered chunks only; not in the paper, which notes that
better schedules exist): QB_CHUNK starts as the first remaining gate's qubits and the pinned
qubits, then grows one pending gate at a time: among the first 512 remaining gates, the first 64
distinct sets of qubits that a gate would add (and that still fit) are tried, and the set with
which a QB_BLOCKED scan of those 512 gates takes the most gates is added (the first such set on a
tie); when nothing fits, the remaining places are filled with qubits by ascending physical bit.

Gathered chunks (``pinned > 0``): the same loop without data movement.  A chunk is any set of c
bits that contains the low ``pinned`` bits; the section gathers it from HBM instead of having
chunk_swap rounds make it contiguous.  QB_CHUNK starts as the pinned qubits and is filled by the
same priority rule; no swap round is emitted and the map stays the identity, so only SWAP
relabels can leave an output reordering.  Each section is ("gblock", chunk_mask, gates).
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class Plan:
    n: int
    c: int
    reserve: int
    restore_layout: bool
    ops: list = field(default_factory=list)  # ("swap"|"unpermute", [(p, q)]) / ("block", [(gi, phys)])
    #                                          / ("gblock", (chunk_mask, [(gi, phys)]))
    final_map: list = field(default_factory=list)  # physical bit of each logical qubit at the end
    pinned: int = 0

    def serialize(self):
        """Integer stream used to compare schedules bit for bit with the library's planner."""
        out = [self.n, self.c, self.reserve, int(self.restore_layout), len(self.ops)]
        for kind, body in self.ops:
            if kind in ("swap", "unpermute"):
                out += [1 if kind == "swap" else 3, len(body)]
                for p, q in body:
                    out += [p, q]
            else:
                if kind == "gblock":
                    mask, body = body
                    out += [4, mask, len(body)]
                else:
                    out += [2, len(body)]
                for gi, phys in body:
                    out += [gi, len(phys), phys[0], phys[1] if len(phys) > 1 else -1]
        out += list(self.final_map)
        return out

    def blocks(self):
        """(chunk bits, gate list) of every section; a contiguous chunk is bits 0..c-1."""
        out = []
        for kind, body in self.ops:
            if kind == "block":
                out.append((list(range(min(self.c, self.n))), body))
            elif kind == "gblock":
                mask, gl = body
                out.append(([b for b in range(self.n) if (mask >> b) & 1], gl))
        return out

    @property
    def n_blocks(self):
        return sum(1 for k, _ in self.ops if k in ("block", "gblock"))

    @property
    def n_swap_rounds(self):
        return sum(1 for k, _ in self.ops if k == "swap")

    @property
    def n_unpermute_rounds(self):
        return sum(1 for k, _ in self.ops if k == "unpermute")


def _canonical_qubits(kind, qubits):
    """Logical qubits of a gate in ascending order (the schedule lists physical bits in this
    order)."""
    return tuple(sorted(qubits))


DIAGONAL_KINDS = ("z", "rz", "cp", "cz")


LOOKAHEAD_WINDOW = 512   # remaining gates a look-ahead scan inspects
LOOKAHEAD_CHOICES = 64   # distinct candidate qubit sets tried per growth step


def _scan_takes(remaining, chosen_set, diag, limit):
    """Number of gates a QB_BLOCKED scan of the first `limit` remaining gates would put in a
    section whose chunk holds `chosen_set` (the scan of the planner loop below, counting only)."""
    blocked, out_blocked, taken = set(), set(), 0
    for gi, qs in remaining[:limit]:
        outside = [q for q in qs if q not in chosen_set]
        if not outside:
            take = not any(q in blocked for q in qs)
        else:
            take = (gi in diag and not any(q in blocked for q in qs if q in chosen_set)
                    and not any(q in out_blocked for q in outside))
        if take:
            taken += 1
        else:
            if any(q in chosen_set for q in qs):
                blocked.update(qs)
            out_blocked.update(outside)
    return taken


def _lookahead_chunk(remaining, target, pinned_qubits, diag, fill_order):
    """QB_CHUNK by look-ahead: the first remaining gate's qubits and the pinned ones, then, step by
    step, the candidate qubit set (new qubits of one of the first LOOKAHEAD_WINDOW remaining
    gates; the first LOOKAHEAD_CHOICES distinct sets that fit) whose scan takes the most gates;
    finally filled in `fill_order`."""
    chosen = set(remaining[0][1]) | set(pinned_qubits)
    while len(chosen) < target:
        best, best_score, tried = None, -1, []
        for _gi, qs in remaining[:LOOKAHEAD_WINDOW]:
            if len(tried) >= LOOKAHEAD_CHOICES:
                break
            fresh = frozenset(qs) - chosen
            if not fresh or len(chosen) + len(fresh) > target or fresh in tried:
                continue
            tried.append(fresh)
            score = _scan_takes(remaining, chosen | fresh, diag, LOOKAHEAD_WINDOW)
            if score > best_score:
                best, best_score = fresh, score
        if best is None:
            break
        chosen |= best
    for q in fill_order:
        if len(chosen) >= target:
            break
        chosen.add(q)
    return chosen


def _rule_chunk(remaining, target, pinned, pinv, n, width):
    """QB_CHUNK by the priority rule (Sec. IV.A with the readings in the module docstring)."""
    chosen, chosen_set = [], set()

    def try_add(qs):
        new = []
        for q in qs:
            if q not in chosen_set and q not in new:
                new.append(q)
        if len(chosen) + len(new) <= target:
            chosen.extend(new)
            chosen_set.update(new)

    for p in range(pinned):  # gathered chunks always hold the low `pinned` bits
        try_add((pinv[p],))
    try_add(remaining[0][1])
    for _gi, qs in remaining:
        if len(chosen) >= target:
            break
        if len(qs) > 1:
            try_add(qs)
    for _gi, qs in remaining:
        if len(chosen) >= target:
            break
        if len(qs) == 1:
            try_add(qs)
    for p in range(n if pinned else width):
        if len(chosen) >= target:
            break
        try_add((pinv[p],))
    return chosen, chosen_set


def plan_blocking(n: int, gates, c: int, reserve: int = 0, restore_layout: bool = True, pinned: int = 0,
                  diag_outside: bool = False, lookahead: bool = False, steer=None, steer_min_chunk: int = 0) -> Plan:
    """`steer` (gathered chunks only): a function that receives, for every section, the candidate
    chunk qubit sets -- the priority rule's chunk, the rule's chunk one and two qubits smaller
    (when at least `steer_min_chunk` (default pinned + 2) and still room for the first remaining
    gate beside the pinned qubits), and the look-ahead chunk, duplicates dropped in that order --
    and returns the index of the one to use.  This is the candidate set a cost model chooses
    from; the choice itself is the caller's."""
    if not (1 <= n <= 62):
        raise ValueError("n out of range")
    if c < 1:
        raise ValueError("c must be >= 1")
    if reserve not in (0, 1):
        raise ValueError("reserve must be 0 or 1")
    width = min(c, n)  # physical bits 0 .. width-1 form a chunk
    target = min(c - reserve, n)
    if target < 1:
        raise ValueError("chunk too small")
    if pinned < 0 or pinned > n or (pinned and target - pinned < 2):
        raise ValueError("pinned bits leave no room for a 2-qubit gate")

    # SWAP gates as relabels: lab[label] = virtual qubit carrying that label.
    lab = list(range(n))
    remaining = []  # (gate index, virtual qubits ascending by label order of description)
    diag = set()    # gates that may join a section with qubits outside its chunk
    for gi, (kind, qubits, _params) in enumerate(gates):
        for q in qubits:
            if not (0 <= q < n):
                raise ValueError(f"gate {gi} qubit {q} out of range")
        if len(set(qubits)) != len(qubits):
            raise ValueError(f"gate {gi} repeats a qubit")
        if kind == "swap":
            a, b = qubits
            lab[a], lab[b] = lab[b], lab[a]
            continue
        vq = tuple(lab[q] for q in _canonical_qubits(kind, qubits))
        if len(vq) > target:
            raise ValueError(f"gate {gi} is wider than the chunk")
        remaining.append((gi, vq))
        if diag_outside and kind in DIAGONAL_KINDS:
            diag.add(gi)

    m = list(range(n))  # virtual (logical) qubit -> physical bit
    pinv = list(range(n))  # physical bit -> virtual qubit
    plan = Plan(n=n, c=c, reserve=reserve, restore_layout=restore_layout, pinned=pinned)

    while remaining:
        # -- choose QB_CHUNK
        if pinned and steer is not None:
            cands = []

            def add(cs):
                if cs not in cands:
                    cands.append(cs)

            add(frozenset(_rule_chunk(remaining, target, pinned, pinv, n, width)[1]))
            min_chunk = steer_min_chunk or pinned + 2
            for d in (1, 2):
                if target - d >= min_chunk and target - d >= len(remaining[0][1]) + pinned:
                    add(frozenset(_rule_chunk(remaining, target - d, pinned, pinv, n, width)[1]))
            add(frozenset(_lookahead_chunk(remaining, target, [pinv[p] for p in range(pinned)], diag,
                                           [pinv[p] for p in range(n)])))
            chosen_set = set(cands[steer(cands)])
            chosen = sorted(chosen_set)
        elif pinned and lookahead:
            chosen_set = _lookahead_chunk(remaining, target, [pinv[p] for p in range(pinned)], diag,
                                          [pinv[p] for p in range(n)])
            chosen = sorted(chosen_set)
        else:
            chosen, chosen_set = _rule_chunk(remaining, target, pinned, pinv, n, width)

        # -- chunk_swap round (none for gathered chunks: the section gathers its bits)
        incoming = [] if pinned else sorted(q for q in chosen if m[q] >= width)
        vacated = sorted(p for p in range(width) if pinv[p] not in chosen_set)
        pairs = []
        for q_in, slot in zip(incoming, vacated):
            old = m[q_in]
            q_out = pinv[slot]
            m[q_in], pinv[slot] = slot, q_in
            m[q_out], pinv[old] = old, q_out
            pairs.append((slot, old))
        if pairs:
            plan.ops.append(("swap", pairs))

        # -- scan REMAINING with QB_BLOCKED
        # diag_outside: a diagonal gate may also take qubits outside the chunk (they are fixed
        # over a chunk), provided no earlier deferred gate touches those qubits
        blocked = set()
        out_blocked = set()
        block = []
        nxt = []
        for gi, qs in remaining:
            outside = [q for q in qs if q not in chosen_set]
            if not outside:
                take = not any(q in blocked for q in qs)
            else:
                take = (gi in diag and not any(q in blocked for q in qs if q in chosen_set)
                        and not any(q in out_blocked for q in outside))
            if take:
                block.append((gi, tuple(m[q] for q in qs)))
            else:
                nxt.append((gi, qs))
                if any(q in chosen_set for q in qs):
                    blocked.update(qs)
                out_blocked.update(outside)
        if pinned:
            mask = 0
            for q in chosen:
                mask |= 1 << m[q]
            plan.ops.append(("gblock", (mask, block)))
        else:
            plan.ops.append(("block", block))
        remaining = nxt

    # -- output reordering: physical bit m[lab[q]] must end at bit q.
    src = [m[lab[q]] for q in range(n)]
    if restore_layout:
        dest = [0] * n
        for q in range(n):
            dest[src[q]] = q
        r1, r2 = [], []
        seen = [False] * n
        for x0 in range(n):
            if seen[x0]:
                continue
            cyc = [x0]
            seen[x0] = True
            y = dest[x0]
            while y != x0:
                cyc.append(y)
                seen[y] = True
                y = dest[y]
            L = len(cyc)
            if L == 1:
                continue
            for i in range(1, (L - 1) // 2 + 1):
                a, b = cyc[i], cyc[L - i]
                r1.append((min(a, b), max(a, b)))
            for i in range(1, L // 2 + 1):
                a, b = cyc[i], cyc[(L + 1 - i) % L]
                r2.append((min(a, b), max(a, b)))
        for r in (r1, r2):
            if r:
                plan.ops.append(("unpermute", sorted(r)))
        plan.final_map = list(range(n))
    else:
        plan.final_map = src
    return plan


def validate(plan: Plan, gates, diag_outside: bool = False) -> None:
    """Raise AssertionError unless the plan is a valid cache-blocked schedule of `gates`:
    every non-SWAP gate is emitted exactly once, every emitted gate's physical bits are in its
    section's chunk (diagonal gates excepted when `diag_outside`), every swap round pairs a bit
    < c with a bit >= c and no bit twice, and the per-qubit gate order of the input is
    preserved."""
    def exempt(gi):
        return diag_outside and gates[gi][0] in DIAGONAL_KINDS
    n, c = plan.n, plan.c
    width = min(c, n)
    emitted = []
    for kind, body in plan.ops:
        if kind == "swap":
            used = set()
            for p, q in body:
                assert p < width <= q < n, (p, q)
                assert p not in used and q not in used
                used.update((p, q))
        elif kind == "unpermute":
            used = set()
            for p, q in body:
                assert 0 <= p < q < n
                assert p not in used and q not in used
                used.update((p, q))
        elif kind == "gblock":
            mask, gl = body
            assert len(gl) > 0, "empty block"
            assert bin(mask).count("1") <= width and mask < (1 << n)
            assert all((mask >> b) & 1 for b in range(plan.pinned)), "pinned bits missing"
            for gi, phys in gl:
                assert exempt(gi) or all((mask >> p) & 1 for p in phys), (phys, mask)
                emitted.append(gi)
        else:
            assert len(body) > 0, "empty block"
            for gi, phys in body:
                assert all(0 <= p < n for p in phys) and (exempt(gi) or all(p < width for p in phys)), phys
                emitted.append(gi)
    expect = [gi for gi, g in enumerate(gates) if g[0] != "swap"]
    assert sorted(emitted) == expect, "each gate exactly once"
    # per-qubit order: for each logical label track positions through relabels
    lab = list(range(n))
    vq_of = {}
    for gi, (kind, qubits, _p) in enumerate(gates):
        if kind == "swap":
            a, b = qubits
            lab[a], lab[b] = lab[b], lab[a]
        else:
            vq_of[gi] = tuple(lab[q] for q in qubits)
    pos = {gi: k for k, gi in enumerate(emitted)}
    last = {}
    for gi in expect:
        for v in vq_of[gi]:
            if v in last:
                assert pos[last[v]] < pos[gi], f"order violated on qubit {v}"
            last[v] = gi

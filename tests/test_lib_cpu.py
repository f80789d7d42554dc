"""Host-side checks of the CUDA library without a GPU: it loads, exports every entry point that
include/sv.h declares, builds gate matrices like the oracle, and its planner's schedules match
the oracle planner bit for bit.  No kernel is launched here."""
import os
import re

import numpy as np
import pytest

import circuitgen as cg
from oracle import gates as og
from oracle import planner, sim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sv():
    from paper_2102_02957_gb300 import build
    build.build()
    import paper_2102_02957_gb300 as m
    m.lib()
    return m


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(sv_[a-z0-9_]+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(sv):
    declared = _declared_functions()
    assert len(declared) >= 20
    lib = sv.lib()
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header(sv):
    declared = set(_declared_functions())
    bound = set(sv._lib.exported_names())
    assert declared == bound, (declared - bound, bound - declared)


KINDS = [("u3", (3,), (0.3, 1.1, -2.0)), ("h", (1,), ()), ("x", (0,), ()), ("y", (2,), ()), ("z", (3,), ()),
         ("ry", (1,), (0.7,)), ("rz", (2,), (1.9,)), ("cx", (3, 1), ()), ("cz", (0, 2), ()),
         ("cp", (1, 3), (0.45,)), ("swap", (0, 3), ())]


@pytest.mark.parametrize("desc", KINDS)
def test_gate_matrices_match_oracle(sv, desc):
    kind, qubits, params = desc
    rec = sv.make_gates([desc])[0]
    order, m = og.matrix_of(kind, qubits, params)
    nq = len(order)
    assert rec["nq"] == nq and tuple(rec["q"][:nq]) == tuple(order)
    got = rec["m"][: 2 * (1 << nq) ** 2].view(np.complex128).reshape(1 << nq, 1 << nq)
    assert np.abs(got - m).max() < 1e-15
    assert bool(rec["flags"] & sv.SV_GATE_SWAP) == (kind == "swap")


def test_unitary_gate_roundtrip(sv):
    rng = np.random.Generator(np.random.PCG64(1))
    u = cg.haar_unitary(rng)
    rec = sv.make_gates([("unitary", (4, 2), (u,))])[0]
    assert tuple(rec["q"]) == (4, 2)
    assert np.array_equal(rec["m"].view(np.complex128).reshape(4, 4), u)


def _gate_one(sv, kind, qubits, params):
    """One record through sv_gate_make (the single-gate entry point)."""
    import ctypes
    rec = np.zeros(1, dtype=sv.GATE_DTYPE)
    q = (ctypes.c_int32 * 2)(*(list(qubits) + [0, 0])[:2])
    if kind == "unitary":
        m = np.ascontiguousarray(params[0], dtype=np.complex128)
        k = sv._lib.SV_K_UNITARY1 if m.shape == (2, 2) else sv._lib.SV_K_UNITARY2
        p = np.ascontiguousarray(m.reshape(-1).view(np.float64))
    else:
        k = sv._KIND[kind]
        p = np.asarray(params, dtype=np.float64) if params else None
    pp = p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if p is not None else None
    sv.check(sv.lib().sv_gate_make(k, q, pp, rec.ctypes.data))
    return rec[0]


def test_gates_make_batch_matches_single_calls(sv):
    """sv_gates_make over a mixed list (every kind, 1- and 2-qubit unitaries) gives the records
    sv_gate_make gives one at a time, and the oracle's matrices."""
    rng = np.random.Generator(np.random.PCG64(5))
    descs = list(KINDS) + [("unitary", (4, 2), (cg.haar_unitary(rng),)),
                           ("unitary", (5,), (np.array([[0, 1j], [1j, 0]]),))] + list(reversed(KINDS))
    recs = sv.make_gates(descs)
    assert len(recs) == len(descs)
    for rec, (kind, qubits, params) in zip(recs, descs):
        one = _gate_one(sv, kind, qubits, params)
        assert rec.tobytes() == one.tobytes(), kind
        if kind != "unitary":
            order, m = og.matrix_of(kind, qubits, params)
            nq = len(order)
            got = rec["m"][: 2 * (1 << nq) ** 2].view(np.complex128).reshape(1 << nq, 1 << nq)
            assert np.abs(got - m).max() < 1e-15
    assert len(sv.make_gates([])) == 0


def test_gates_make_batch_errors(sv):
    L = sv.lib()
    out = np.zeros(3, dtype=sv.GATE_DTYPE)
    kinds = np.array([sv._KIND["h"], sv._KIND["cx"], sv._KIND["u3"]], dtype=np.int32)
    qubits = np.array([[0, 0], [1, 1], [2, 0]], dtype=np.int32)  # gate 1 repeats a qubit
    params = np.zeros((3, 32))
    st = L.sv_gates_make(3, kinds.ctypes.data, qubits.ctypes.data, params.ctypes.data, 32, out.ctypes.data)
    assert st == sv._lib.SV_ERR_ARG and "gate 1" in L.sv_last_error().decode()
    assert out[0]["nq"] == 1 and out[2]["nq"] == 0  # entries before the failing one are written, later ones not
    qubits[1] = (1, 2)
    # a stride too short for U3's three angles, and parameters missing altogether
    assert L.sv_gates_make(3, kinds.ctypes.data, qubits.ctypes.data, params.ctypes.data, 2, out.ctypes.data) \
        == sv._lib.SV_ERR_ARG and "gate 2" in L.sv_last_error().decode()
    assert L.sv_gates_make(3, kinds.ctypes.data, qubits.ctypes.data, None, 32, out.ctypes.data) == sv._lib.SV_ERR_ARG
    assert L.sv_gates_make(2, kinds.ctypes.data, qubits.ctypes.data, None, 0, out.ctypes.data) == sv._lib.SV_OK
    assert L.sv_gates_make(-1, kinds.ctypes.data, qubits.ctypes.data, None, 0, out.ctypes.data) == sv._lib.SV_ERR_ARG
    assert L.sv_gates_make(1, None, qubits.ctypes.data, None, 0, out.ctypes.data) == sv._lib.SV_ERR_ARG
    bad = np.array([99], dtype=np.int32)
    assert L.sv_gates_make(1, bad.ctypes.data, qubits.ctypes.data, None, 0, out.ctypes.data) == sv._lib.SV_ERR_ARG


def _circuits(n, seed):
    return [cg.random_layers(n, 4, seed), cg.quantum_volume(n, 4, seed), cg.qft(n), cg.hea(n, 2, seed, 1),
            cg.noisy_trajectory(n, 3, 0.3, seed, 2), cg.mirror(cg.quantum_volume(n, 2, seed + 1))]


@pytest.mark.parametrize("n", [4, 7, 12, 16, 30])
@pytest.mark.parametrize("c", [2, 4, 6, 10, 13])
def test_planner_schedule_parity(sv, n, c):
    for reserve in (0, 1):
        if c - reserve < 2:
            continue
        for restore in (True, False):
            for desc in _circuits(n, 3 * n + c):
                gates = sv.make_gates(desc)
                p = sv.Plan(n, gates, chunk_bits=c, reserve=reserve, restore_layout=restore)
                q = planner.plan_blocking(n, desc, c, reserve, restore)
                assert p.serialize() == q.serialize()
                inf = p.info()
                assert inf.n_blocks == q.n_blocks and inf.n_swap_rounds == q.n_swap_rounds
                assert list(inf.final_map[:n]) == q.final_map


def test_planner_full_size_workloads(sv):
    for name in ("qv30", "rl28", "qft28", "rl16", "qv32"):
        w = cg.WORKLOADS[name]
        desc = cg.build(name)
        p = sv.Plan(w["n"], sv.make_gates(desc), chunk_bits=w["c"])
        q = planner.plan_blocking(w["n"], desc, w["c"])
        assert p.serialize() == q.serialize(), name


def test_planner_errors(sv):
    gates = sv.make_gates([("cx", (0, 1), ())])
    with pytest.raises(sv.SVError) as e:
        sv.Plan(4, gates, chunk_bits=2, reserve=1)
    assert e.value.status == sv._lib.SV_ERR_ARG
    bad = gates.copy()
    bad[0]["q"][0] = 9
    with pytest.raises(sv.SVError):
        sv.Plan(4, bad, chunk_bits=3)
    with pytest.raises(sv.SVError):
        sv.make_gates([("cx", (1, 1), ())])


@pytest.mark.parametrize("n,c,pinned", [(6, 4, 1), (12, 8, 3), (16, 10, 4), (30, 13, 4), (30, 13, 3)])
def test_planner_schedule_parity_gathered(sv, n, c, pinned):
    for desc in _circuits(n, 7 * n + c):
        gates = sv.make_gates(desc)
        p = sv.Plan(n, gates, chunk_bits=c, gather_pinned=pinned)
        q = planner.plan_blocking(n, desc, c, pinned=pinned)
        assert p.serialize() == q.serialize()
        assert p.info().n_swap_rounds == 0


def test_binding_constants_match_header():
    """Every enumerator `SV_NAME = value` in include/sv.h has the same value in the binding."""
    import re
    from paper_2102_02957_gb300 import _lib
    with open(os.path.join(ROOT, "include", "sv.h")) as f:
        text = f.read()
    found = dict((k, int(v)) for k, v in re.findall(r"\b(SV_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert "SV_BATCH_FROM_ZERO" in found and "SV_ERR_TIMEOUT" in found
    for name, value in found.items():
        if hasattr(_lib, name):
            assert getattr(_lib, name) == value, name


def test_section_features_hand_computed():
    """Cost-model features of a one-section plan, worked out by hand (host code, no GPU)."""
    import paper_2102_02957_gb300 as sv
    desc = [("h", (0,), ()), ("cx", (0, 1), ()), ("cz", (2, 3), ())]
    g = sv.make_gates(desc)
    plan = sv.Plan(8, g, chunk_bits=6, gather_pinned=4)
    f = plan.features(g, "c64")
    assert f.shape == (1, 16)
    want = np.array([6 / 16, 4 / 8, np.log2(4) / 10, np.log2(2) / 6,
                     2 / 5, 1 / 5, 1 / 5, 1 / 5, 0, 0,        # qubit positions 0,0,1,2,3
                     2 / 3, 2 / 3, 0, 8 / 32, 0, 1], dtype=np.float32)
    np.testing.assert_allclose(f[0], want, rtol=1e-6, atol=1e-7)
    f128 = plan.features(g, "c128")
    assert f128[0, 12] == 1.0


@pytest.mark.parametrize("n,c,pinned", [(8, 3, 0), (12, 6, 0), (16, 10, 0), (12, 8, 4), (16, 10, 3), (30, 13, 4),
                                        (28, 12, 0)])
def test_planner_schedule_parity_diag_outside(sv, n, c, pinned):
    """Both planners take the same diagonal gates into sections with qubits outside the chunk."""
    import math
    rng = np.random.Generator(np.random.PCG64(n * 100 + c))
    mixed = []
    for g in cg.random_layers(n, 3, n + c):
        mixed.append(g)
        a, b = (int(v) for v in rng.permutation(n)[:2])
        mixed.append([("cz", (a, b), ()), ("cp", (a, b), (0.7,)), ("rz", (a,), (1.3,)), ("z", (b,), ())][int(rng.integers(0, 4))])
    for desc in [cg.qft(n), cg.hea(n, 2, 3, 1), mixed] + _circuits(n, n + c):
        gates = sv.make_gates(desc)
        p = sv.Plan(n, gates, chunk_bits=c, gather_pinned=pinned, diag_outside=1)
        q = planner.plan_blocking(n, desc, c, pinned=pinned, diag_outside=True)
        assert p.serialize() == q.serialize()
    qft = cg.qft(n)
    p = sv.Plan(n, sv.make_gates(qft), chunk_bits=c, gather_pinned=pinned, diag_outside=1)
    assert p.info().n_blocks == math.ceil((n - pinned) / (c - pinned))


def _plan_from_stream(stream, pinned):
    """The library's serialised schedule as an oracle Plan (same integer format)."""
    it = iter(stream)
    n, c, reserve, restore, nops = (next(it) for _ in range(5))
    plan = planner.Plan(n=n, c=c, reserve=reserve, restore_layout=bool(restore), pinned=pinned)
    for _ in range(nops):
        kind = next(it)
        if kind in (1, 3):
            cnt = next(it)
            plan.ops.append(("swap" if kind == 1 else "unpermute", [(next(it), next(it)) for _ in range(cnt)]))
        else:
            mask = next(it) if kind == 4 else None
            cnt = next(it)
            body = []
            for _ in range(cnt):
                gi, nq, p0, p1 = next(it), next(it), next(it), next(it)
                body.append((gi, (p0,) if nq == 1 else (p0, p1)))
            plan.ops.append(("gblock", (mask, body)) if kind == 4 else ("block", body))
    plan.final_map = list(it)
    return plan


@pytest.mark.parametrize("n,c,pinned", [(6, 4, 1), (8, 5, 1), (10, 6, 2), (12, 8, 4), (14, 9, 3), (16, 10, 4),
                                        (30, 12, 5), (30, 13, 4)])
def test_planner_schedule_parity_lookahead(sv, n, c, pinned):
    """The look-ahead chunk choice: the library's schedules equal the oracle's restatement bit for
    bit, with and without diagonal gates outside the chunk."""
    for desc in _circuits(n, 11 * n + c):
        gates = sv.make_gates(desc)
        for diag in (0, 1):
            p = sv.Plan(n, gates, chunk_bits=c, gather_pinned=pinned, lookahead=1, diag_outside=diag)
            q = planner.plan_blocking(n, desc, c, pinned=pinned, lookahead=True, diag_outside=bool(diag))
            assert p.serialize() == q.serialize(), (n, c, pinned, diag)


@pytest.mark.parametrize("name,c,pinned", [("qv30", 12, 5), ("qv32", 13, 4), ("rl28", 12, 5), ("qft28", 12, 4),
                                           ("rl32", 13, 4)])
def test_planner_schedule_parity_lookahead_full_size(sv, name, c, pinned):
    """The schedules behind the benchmark (quantum volume n = 30, chunk 12 with 5 pinned bits) and
    the other full-size workloads, look-ahead chunk choice, against the oracle bit for bit."""
    w = cg.WORKLOADS[name]
    desc = cg.build(name)
    gates = sv.make_gates(desc)
    for diag in (0, 1):
        p = sv.Plan(w["n"], gates, chunk_bits=c, gather_pinned=pinned, lookahead=1, diag_outside=diag)
        q = planner.plan_blocking(w["n"], desc, c, pinned=pinned, lookahead=True, diag_outside=bool(diag))
        assert p.serialize() == q.serialize(), (name, diag)


@pytest.mark.parametrize("n,c,pinned", [(10, 6, 2), (12, 8, 4), (14, 9, 3)])
def test_lookahead_plans_valid_and_equivalent(sv, n, c, pinned):
    """The look-ahead chunk choice (a heuristic of this library, not the paper's rule) yields valid
    schedules that simulate to the original circuit, with no more sections than the rule on
    these circuits (no GPU)."""
    for desc in _circuits(n, 5 * n + c):
        gates = sv.make_gates(desc)
        for diag in (0, 1):
            p = sv.Plan(n, gates, chunk_bits=c, gather_pinned=pinned, lookahead=1, diag_outside=diag)
            q = _plan_from_stream(p.serialize(), pinned)
            planner.validate(q, desc, diag_outside=bool(diag))
            ref = sim.simulate(n, desc, 3)
            assert np.abs(sim.execute_plan(n, desc, q, 3) - ref).max() < 1e-12
    qv = cg.quantum_volume(n, 8, n)
    g = sv.make_gates(qv)
    assert (sv.Plan(n, g, chunk_bits=c, gather_pinned=pinned, lookahead=1).info().n_blocks
            <= sv.Plan(n, g, chunk_bits=c, gather_pinned=pinned).info().n_blocks)


@pytest.mark.parametrize("seg_bits", [3, 4, 5])
def test_plan_widths_default_to_the_plan(sv, seg_bits):
    """Plans made without a cost model give every section the plan's register-group width; the
    group count of the plan info is the sum of the per-section beam-search groups, which never
    exceeds one group per gate."""
    n = 22
    g = sv.make_gates(cg.quantum_volume(n, 10, 5))
    plan = sv.Plan(n, g, chunk_bits=12, gather_pinned=5, use_tc=1, seg_bits=seg_bits, lookahead=1)
    w = plan.widths()
    inf = plan.info()
    assert len(w) == inf.n_blocks and set(int(x) for x in w) == {seg_bits}
    assert inf.n_blocks <= inf.n_segments <= inf.n_gates_emitted


def _greedy_groups(masks, r):
    """Register groups by greedy growth (the first pending gate's bits, then the pending gate,
    among the first 64 with new bits, that lets the group take the most gates)."""
    pending = list(range(len(masks)))

    def split(pend, bits):
        blocked, rest = 0, []
        for i in pend:
            if (masks[i] & ~bits) == 0 and (masks[i] & blocked) == 0:
                continue
            blocked |= masks[i]
            rest.append(i)
        return rest

    groups = 0
    while pending:
        s = masks[pending[0]]
        while bin(s).count("1") < r:
            best, best_k, tried = 0, -1, 0
            for i in pending:
                fresh = masks[i] & ~s
                if not fresh or bin(s | fresh).count("1") > r:
                    continue
                tried += 1
                if tried > 64:
                    break
                k = len(pending) - len(split(pending, s | fresh))
                if k > best_k:
                    best_k, best = k, fresh
            if not best:
                break
            s |= best
        pending = split(pending, s)
        groups += 1
    return groups


@pytest.mark.parametrize("name,c,pinned", [("qv30", 12, 5), ("qv26", 12, 5), ("rl28", 12, 4)])
def test_register_group_search_bounds(sv, name, c, pinned):
    """The library's register groups per plan (beam search) never outnumber greedy growth's
    (restated here) and never undercut the lower bound ceil(bits in use / r) of any section."""
    w = cg.WORKLOADS[name]
    desc = cg.build(name)
    n = w["n"]
    lib_plan = sv.Plan(n, sv.make_gates(desc), chunk_bits=c, gather_pinned=pinned, lookahead=1)
    oracle_plan = planner.plan_blocking(n, desc, c, pinned=pinned, lookahead=True)
    greedy = bound = 0
    for bits, gl in oracle_plan.blocks():
        masks = []
        for _gi, phys in gl:
            m = 0
            for q in phys:
                if q >= 0:
                    m |= 1 << q
            masks.append(m)
        greedy += _greedy_groups(masks, 4)
        used = 0
        for m in masks:
            used |= m
        bound += -(-bin(used).count("1") // 4)
    got = lib_plan.info().n_segments
    print(f"{name}: beam {got}, greedy {greedy}, lower bound {bound}")
    assert bound <= got <= greedy


def _beam_groups(masks, r, width, budget=4_000_000):
    """Register groups by beam search, written out plainly: level by level every r-subset of the
    bits the pending gates use (lexicographic in bit position) is tried on every kept pending
    list; a child that takes at least one gate and whose pending list was not produced before on
    this level is kept; children are ranked by ceil(bits used / r), then pending gates, then bits
    used, ties in the order found; the best `width` survive; the first subset that empties a
    list, or a list whose bits fit one group, ends the search.  None once the budget (the pending
    list's length per subset tried) is spent."""
    from itertools import combinations

    def split(pend, bits):
        blocked, rest = 0, []
        for i in pend:
            if (masks[i] & ~bits) == 0 and (masks[i] & blocked) == 0:
                continue
            blocked |= masks[i]
            rest.append(i)
        return rest

    def used_of(pend):
        u = 0
        for i in pend:
            u |= masks[i]
        return u

    if not masks:
        return 0
    beam = [(list(range(len(masks))), 0)]  # (pending list, groups so far)
    while True:
        children, seen = [], set()
        for pend, ngroups in beam:
            used = used_of(pend)
            if bin(used).count("1") <= r:
                return ngroups + 1
            bits = [b for b in range(64) if (used >> b) & 1]
            for sub in combinations(bits, r):
                budget -= len(pend)
                if budget < 0:
                    return None
                rest = split(pend, sum(1 << b for b in sub))
                if not rest:
                    return ngroups + 1
                if len(rest) < len(pend) and tuple(rest) not in seen:
                    seen.add(tuple(rest))
                    nbits = bin(used_of(rest)).count("1")
                    children.append(((-(-nbits // r), len(rest), nbits), rest, ngroups + 1))
        children.sort(key=lambda ch: ch[0])  # stable: ties keep the order found
        beam = [(rest, ng) for _key, rest, ng in children[:width]]


@pytest.mark.parametrize("name,c", [("qv26", 12), ("rl16", 10), ("qft28", 12), ("rl28", 12), ("qv30", 12)])
def test_register_group_search_matches_restatement(sv, name, c):
    """The library's register-group count (paper layout: chunk bits 0..c-1, 4-bit groups) equals
    the plain beam search above section by section, summed over the plan (beam of 8 for sections
    of up to 32 gates, of 1 above; greedy growth where the search runs out of budget)."""
    w = cg.WORKLOADS[name]
    desc = cg.build(name)
    n = w["n"]
    lib_plan = sv.Plan(n, sv.make_gates(desc), chunk_bits=c)
    oracle_plan = planner.plan_blocking(n, desc, c)
    total = 0
    for _bits, gl in oracle_plan.blocks():
        masks = []
        for _gi, phys in gl:
            m = 0
            for q in phys:
                if 0 <= q < c:
                    m |= 1 << q
            masks.append(m)
        got = _beam_groups(masks, min(4, c, n), 8 if len(masks) <= 32 else 1)
        total += got if got is not None else _greedy_groups(masks, min(4, c, n))
    assert lib_plan.info().n_segments == total


def test_plan_widths_arguments(sv):
    """sv_plan_get_widths: null plan or count and a negative capacity are argument errors; a
    capacity smaller than the section count fills what fits and still reports the count."""
    import ctypes
    lib = sv._lib.lib()
    g = sv.make_gates(cg.quantum_volume(12, 4, 2))
    plan = sv.Plan(12, g, chunk_bits=8, gather_pinned=4, use_tc=0)
    cnt = ctypes.c_int64()
    assert lib.sv_plan_get_widths(None, None, 0, ctypes.byref(cnt)) == sv._lib.SV_ERR_ARG
    assert lib.sv_plan_get_widths(plan.handle, None, 0, None) == sv._lib.SV_ERR_ARG
    assert lib.sv_plan_get_widths(plan.handle, None, -1, ctypes.byref(cnt)) == sv._lib.SV_ERR_ARG
    out = (ctypes.c_int32 * 1)(-7)
    assert lib.sv_plan_get_widths(plan.handle, out, 1, ctypes.byref(cnt)) == sv._lib.SV_OK
    assert cnt.value == plan.info().n_blocks >= 1 and out[0] == 4

"""Pins for the oracle's cache-blocking planner (Sec. IV.A Listing 3, Sec. IV.C Fig. 10), no GPU.

The paper's worked example (Fig. 9) is an unavailable image, so the swap count is parity
unpinned; the schedule is pinned by a hand-worked example, validity and simulation
equivalence."""
import itertools
import math
import os

import numpy as np
import pytest

import circuitgen as cg
from oracle import planner, sim


def _read_plan_golden(path):
    ops, meta = [], {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "op":
                kind = parts[1]
                if kind in ("swap", "unpermute"):
                    ops.append((kind, [tuple(int(v) for v in p.split(",")) for p in parts[2:]]))
                else:
                    body = []
                    for p in parts[2:]:
                        gi, phys = p.split(":")
                        body.append((int(gi), tuple(int(v) for v in phys.split(","))))
                    ops.append(("block", body))
            else:
                meta[parts[0]] = parts[1:]
    gates = []
    for g in meta["gates"]:
        kind, qs = g.split(":")
        gates.append((kind, tuple(int(v) for v in qs.split(",")), ()))
    return int(meta["n"][0]), int(meta["c"][0]), gates, ops


def test_hand_worked_schedule(golden_dir):
    n, c, gates, ops = _read_plan_golden(os.path.join(golden_dir, "planner_n4_c2.txt"))
    p = planner.plan_blocking(n, gates, c)
    assert p.ops == ops
    assert p.final_map == list(range(n))


def _circuits(n, seed):
    return [
        cg.random_layers(n, 4, seed),
        cg.quantum_volume(n, 4, seed),
        cg.qft(n),
        cg.qft(n, with_swaps=False),
        cg.hea(n, 2, seed, 0),
        cg.noisy_trajectory(n, 3, 0.2, seed, 1),
    ]


@pytest.mark.parametrize("n,c", [(4, 2), (5, 3), (7, 4), (8, 8), (9, 3), (10, 6), (12, 5), (6, 12)])
@pytest.mark.parametrize("reserve", [0, 1])
def test_validity_and_equivalence(n, c, reserve):
    if c - reserve < 2:
        pytest.skip("chunk narrower than a 2-qubit gate")
    for i, gates in enumerate(_circuits(n, 10 * n + c)):
        p = planner.plan_blocking(n, gates, c, reserve=reserve)
        planner.validate(p, gates)
        ref = sim.simulate(n, gates, 5 % (1 << n))
        got = sim.execute_plan(n, gates, p, 5 % (1 << n))
        assert np.abs(ref - got).max() < 1e-12, (i, n, c)


@pytest.mark.parametrize("n,c", [(6, 3), (9, 4), (11, 5)])
def test_keep_layout_map(n, c):
    gates = cg.random_layers(n, 3, 7) + [("swap", (0, n - 1), ())] + cg.quantum_volume(n, 2, 8)
    p_keep = planner.plan_blocking(n, gates, c, restore_layout=False)
    planner.validate(p_keep, gates)
    assert p_keep.n_unpermute_rounds == 0
    got = sim.execute_plan(n, gates, p_keep, 3)
    # logical qubit q sits on physical bit final_map[q]: gather it back
    idx = np.arange(1 << n)
    phys = np.zeros_like(idx)
    for q in range(n):
        phys |= ((idx >> q) & 1) << p_keep.final_map[q]
    ref = sim.simulate(n, gates, 3)
    assert np.abs(got[phys] - ref).max() < 1e-12


def test_no_swaps_when_state_fits_chunk():
    gates = cg.random_layers(6, 5, 1)
    p = planner.plan_blocking(6, gates, 10)
    assert p.n_swap_rounds == 0 and p.n_blocks == 1 and p.n_unpermute_rounds == 0


def test_unpermute_is_at_most_two_rounds_and_restores():
    # any final bit permutation is undone by <= 2 rounds of disjoint transpositions
    n = 7
    for perm in itertools.islice(itertools.permutations(range(n)), 0, 5040, 97):
        gates = []
        # build the permutation from SWAP relabels (bubble sort)
        cur = list(range(n))
        target = list(perm)
        for i in range(n):
            j = cur.index(target[i])
            while j > i:
                gates.append(("swap", (j - 1, j), ()))
                cur[j - 1], cur[j] = cur[j], cur[j - 1]
                j -= 1
        gates.append(("h", (0,), ()))
        p = planner.plan_blocking(n, gates, 3)
        assert p.n_unpermute_rounds <= 2
        ref = sim.simulate(n, gates, 77)
        assert np.abs(sim.execute_plan(n, gates, p, 77) - ref).max() < 1e-13


def test_first_gate_always_progresses():
    # every iteration emits at least the first remaining gate -> blocks never empty
    gates = cg.quantum_volume(10, 6, 3)
    p = planner.plan_blocking(10, gates, 2)
    assert all(len(b) >= 1 for k, b in p.ops if k == "block")
    assert p.n_blocks <= len(gates)


def test_gate_wider_than_chunk_rejected():
    with pytest.raises(ValueError):
        planner.plan_blocking(5, [("cx", (0, 1), ())], 2, reserve=1)


def test_swap_counts_shrink_with_bigger_chunks():
    gates = cg.quantum_volume(16, 10, 2)
    counts = [planner.plan_blocking(16, gates, c).n_swap_rounds for c in (4, 8, 12, 16)]
    assert counts == sorted(counts, reverse=True) and counts[-1] == 0


@pytest.mark.parametrize("n,c,pinned", [(6, 4, 1), (9, 5, 2), (10, 6, 4), (12, 8, 3), (12, 12, 4), (7, 9, 2)])
def test_gathered_chunks_validity_and_equivalence(n, c, pinned):
    for gates in _circuits(n, 5 * n + c + pinned):
        p = planner.plan_blocking(n, gates, c, pinned=pinned)
        planner.validate(p, gates)
        assert p.n_swap_rounds == 0
        for bits, _ in p.blocks():
            assert set(range(pinned)) <= set(bits) and len(bits) <= min(c, n)
        ref = sim.simulate(n, gates, 7 % (1 << n))
        assert np.abs(sim.execute_plan(n, gates, p, 7 % (1 << n)) - ref).max() < 1e-12


def test_gathered_chunks_need_room():
    with pytest.raises(ValueError):
        planner.plan_blocking(8, [("cx", (0, 5), ())], 4, pinned=3)


def _diag_circuits(n, seed):
    """Circuits rich in diagonal gates: QFT (CP), a CZ ladder ansatz, random layers with CZ/CP/RZ/Z
    sprinkled in."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mixed = []
    for g in cg.random_layers(n, 3, seed):
        mixed.append(g)
        if rng.random() < 0.5:
            a, b = (int(v) for v in rng.permutation(n)[:2])
            r = int(rng.integers(0, 4))
            mixed.append([("cz", (a, b), ()), ("cp", (a, b), (float(rng.uniform(0, 6.3)),)),
                          ("rz", (a,), (float(rng.uniform(0, 6.3)),)), ("z", (b,), ())][r])
    return [cg.qft(n), cg.hea(n, 3, seed, 0), mixed]


@pytest.mark.parametrize("n,c,pinned", [(8, 3, 0), (10, 4, 0), (12, 6, 0), (10, 6, 3), (12, 8, 4), (9, 4, 1)])
def test_diag_outside_validity_and_equivalence(n, c, pinned):
    """Diagonal gates that join a section with qubits outside its chunk: the schedule stays valid
    (every other gate inside its chunk, per-qubit order kept) and simulates to the same state."""
    for gates in _diag_circuits(n, 11 * n + c):
        p = planner.plan_blocking(n, gates, c, pinned=pinned, diag_outside=True)
        planner.validate(p, gates, diag_outside=True)
        ref = sim.simulate(n, gates, 5 % (1 << n))
        assert np.abs(sim.execute_plan(n, gates, p, 5 % (1 << n)) - ref).max() < 1e-12
        base = planner.plan_blocking(n, gates, c, pinned=pinned)
        assert p.n_blocks <= base.n_blocks


def test_diag_outside_qft_needs_one_section_per_chunk_of_hadamards():
    """In the QFT every gate but the n Hadamards is a controlled phase, so with diag_outside a
    section takes the Hadamards of its chunk qubits and every phase that touches them: the number
    of sections is ceil(n / free chunk bits) with gathered chunks (here 16 qubits, chunk 8 with 2
    pinned bits -> 6 free -> 3 sections), against one section per few Hadamards otherwise."""
    gates = cg.qft(16)
    for n, c, pinned in ((16, 8, 2), (16, 8, 0), (16, 5, 1)):
        p = planner.plan_blocking(n, gates, c, pinned=pinned, diag_outside=True)
        base = planner.plan_blocking(n, gates, c, pinned=pinned)
        assert p.n_blocks == math.ceil((n - pinned) / (c - pinned)), (c, pinned, p.n_blocks)
        assert p.n_blocks < base.n_blocks


def test_lookahead_hand_worked_example():
    """Look-ahead chunk choice on a case worked out by hand (n = 8, chunk of 5 qubits, qubit 0
    pinned).  Gates: g0 = CX(1,2), g1 = CX(3,4), g2..g5 = CX(5,6).
    Rule (Sec. IV.A priority): {0} + g0's {1,2} + the next multi-qubit gate that fits, g1's {3,4}
    -> section 1 takes g0, g1; section 2 starts {0} + {5,6} and fills by ascending bit 1, 2.
    Look-ahead: start {0,1,2}; candidate {3,4} lets a QB_BLOCKED scan take g0, g1 (2 gates),
    candidate {5,6} takes g0, g2, g3, g4, g5 (5 gates; g1 is deferred without blocking anything)
    -> section 1 = {0,1,2,5,6} with g0, g2..g5; section 2 = {0,3,4} filled with 1, 2."""
    desc = [("cx", (1, 2), ()), ("cx", (3, 4), ())] + [("cx", (5, 6), ())] * 4
    la = planner.plan_blocking(8, desc, 5, pinned=1, lookahead=True)
    assert la.ops == [
        ("gblock", (0b1100111, [(0, (1, 2)), (2, (5, 6)), (3, (5, 6)), (4, (5, 6)), (5, (5, 6))])),
        ("gblock", (0b0011111, [(1, (3, 4))])),
    ]
    rule = planner.plan_blocking(8, desc, 5, pinned=1)
    assert rule.ops == [
        ("gblock", (0b0011111, [(0, (1, 2)), (1, (3, 4))])),
        ("gblock", (0b1100111, [(2, (5, 6)), (3, (5, 6)), (4, (5, 6)), (5, (5, 6))])),
    ]


@pytest.mark.parametrize("n,c,pinned", [(8, 5, 1), (10, 6, 2), (12, 8, 4), (14, 9, 3)])
def test_lookahead_plans_valid_and_equivalent_oracle(n, c, pinned):
    """The oracle's own look-ahead schedules: valid, and simulating them (sections on their
    chunk bits, then the reordering) gives the original circuit's state."""
    rng_seed = 31 * n + c
    circuits = [cg.random_layers(n, 4, rng_seed), cg.quantum_volume(n, 5, rng_seed), cg.qft(n),
                cg.hea(n, 2, rng_seed, 1), cg.noisy_trajectory(n, 3, 0.3, rng_seed, 2)]
    for desc in circuits:
        for diag in (False, True):
            plan = planner.plan_blocking(n, desc, c, pinned=pinned, lookahead=True, diag_outside=diag)
            planner.validate(plan, desc, diag_outside=diag)
            ref = sim.simulate(n, desc, 3)
            assert np.abs(sim.execute_plan(n, desc, plan, 3) - ref).max() < 1e-12

"""The seeded input recipes (circuitgen) against what they are stated to draw: gate counts and
structure of every named workload, Haar-distributed SU(4) gates, the depolarizing insertion rate
and the uniformity of the inserted Pauli words, and the batch composition.  No GPU, no oracle."""
import math

import numpy as np
import pytest

import circuitgen as cg


@pytest.mark.parametrize("name,gates,swaps", [("rl16", 480, 0), ("qft28", 406 + 14, 14), ("rl28", 1680, 0),
                                              ("qv30", 450, 0), ("qv26", 130, 0), ("rl32", 1536, 0),
                                              ("qv32", 512, 0)])
def test_workload_sizes(name, gates, swaps):
    desc = cg.build(name)
    assert len(desc) == gates
    assert sum(1 for k, _q, _p in desc if k == "swap") == swaps
    n = cg.WORKLOADS[name]["n"]
    assert all(0 <= q < n for _k, qs, _p in desc for q in qs)


@pytest.mark.parametrize("n", [5, 8, 13])
def test_random_layers_structure(n):
    depth = 6
    desc = cg.random_layers(n, depth, 3)
    per = n + n // 2
    assert len(desc) == depth * per
    for layer in range(depth):
        body = desc[layer * per:(layer + 1) * per]
        assert [g[1] for g in body[:n]] == [(q,) for q in range(n)]
        assert all(g[0] == "u3" and all(0.0 <= a < 2 * math.pi for a in g[2]) for g in body[:n])
        pairs = [g[1] for g in body[n:]]
        assert all(g[0] == "cx" for g in body[n:])
        used = [q for p in pairs for q in p]
        assert len(set(used)) == len(used) == 2 * (n // 2)  # a matching: no qubit twice


def test_random_layer_angles_uniform():
    ang = np.array([a for g in cg.random_layers(16, 40, 9) if g[0] == "u3" for a in g[2]])
    # Kolmogorov-Smirnov distance to U[0, 2pi) for 1920 draws: 1.63/sqrt(N) is the 1 % level
    x = np.sort(ang / (2 * math.pi))
    k = np.arange(1, len(x) + 1) / len(x)
    d = max(np.max(k - x), np.max(x - (k - 1.0 / len(x))))
    assert d < 1.63 / math.sqrt(len(x))


@pytest.mark.parametrize("n", [6, 9, 30])
def test_quantum_volume_structure(n):
    depth = 4
    desc = cg.quantum_volume(n, depth, 5)
    assert len(desc) == depth * (n // 2)
    for layer in range(depth):
        body = desc[layer * (n // 2):(layer + 1) * (n // 2)]
        used = [q for g in body for q in g[1]]
        assert len(set(used)) == len(used)
        for kind, _qs, (u,) in body:
            assert kind == "unitary" and u.shape == (4, 4)
            assert np.abs(u.conj().T @ u - np.eye(4)).max() < 1e-13
            assert abs(np.linalg.det(u) - 1.0) < 1e-12


def test_haar_su4_moments():
    """Haar measure on SU(4): E[tr U] = 0, E[|tr U|^2] = 1, E[|U00|^2] = 1/4, E[|U00|^4] = 1/10.
    QR of a Ginibre matrix without moving R's diagonal phases into Q gives E[|tr U|^2] near 1.86,
    so the second moment of the trace tells the two apart."""
    rng = np.random.Generator(np.random.PCG64(21))
    N = 6000
    us = [cg.haar_unitary(rng) for _ in range(N)]
    tr = np.array([np.trace(u) for u in us])
    t2 = np.abs(tr) ** 2
    u00 = np.array([abs(u[0, 0]) ** 2 for u in us])
    se = 1.0 / math.sqrt(N)
    assert abs(tr.mean()) < 5 * se
    assert abs(t2.mean() - 1.0) < 5 * t2.std() * se
    assert abs(u00.mean() - 0.25) < 5 * u00.std() * se
    assert abs((u00 ** 2).mean() - 0.1) < 5 * (u00 ** 2).std() * se


def test_noisy_trajectory_insertion_rate_and_words():
    """After each gate a Pauli word is inserted with probability p, uniform over the 3 (1-qubit
    gate) or 15 (2-qubit gate) non-identity words; the trajectory keeps the base circuit."""
    n, depth, p = 12, 30, 0.25
    base = cg.random_layers(n, depth, 7 * 1000003 + n)
    inserted, words1, words2 = 0, {}, {}
    trials = 0
    for t in range(40):
        traj = cg.noisy_trajectory(n, depth, p, 7, t)
        i = 0
        for g in base:
            assert traj[i] == g
            i += 1
            trials += 1
            word = []
            while i < len(traj) and traj[i][0] in ("x", "y", "z") and traj[i][1][0] in g[1] and \
                    (not word or traj[i][1][0] != word[-1][1]):
                word.append((traj[i][0], traj[i][1][0]))
                i += 1
            if word:
                inserted += 1
                key = tuple(next((k for k, q in word if q == qq), "i") for qq in g[1])
                (words1 if len(g[1]) == 1 else words2)[key] = (words1 if len(g[1]) == 1 else words2).get(key, 0) + 1
        assert i == len(traj)
    # binomial count of insertions
    assert abs(inserted - p * trials) < 5 * math.sqrt(trials * p * (1 - p))
    # uniform words: chi-square at the 0.1 % level (df 2: 13.8, df 14: 36.1)
    for words, kinds, crit in ((words1, 3, 13.8), (words2, 15, 36.1)):
        assert len(words) == kinds
        tot = sum(words.values())
        chi2 = sum((c - tot / kinds) ** 2 / (tot / kinds) for c in words.values())
        assert chi2 < crit, (kinds, chi2)
        assert all(k != ("i",) * len(k) for k in words)


def test_hea_structure():
    n, layers = 7, 3
    desc = cg.hea(n, layers, 8, 2)
    per = n + (n - 1)
    assert len(desc) == layers * per + n
    for layer in range(layers):
        body = desc[layer * per:(layer + 1) * per]
        assert [(g[0], g[1]) for g in body[:n]] == [("ry", (q,)) for q in range(n)]
        assert [(g[0], g[1]) for g in body[n:]] == [("cz", (q, q + 1)) for q in range(n - 1)]
    assert [(g[0], g[1]) for g in desc[-n:]] == [("ry", (q,)) for q in range(n)]
    assert all(0.0 <= g[2][0] < 2 * math.pi for g in desc if g[0] == "ry")
    assert cg.hea(n, layers, 8, 2) == desc and cg.hea(n, layers, 8, 3) != desc


def test_qft_structure():
    n = 6
    desc = cg.qft(n)
    assert [g for g in desc if g[0] == "h"] == [("h", (j,), ()) for j in range(n - 1, -1, -1)]
    cps = [g for g in desc if g[0] == "cp"]
    assert len(cps) == n * (n - 1) // 2
    for _k, (m, j), (phi,) in cps:
        assert m < j and phi == math.pi / (1 << (j - m))
    assert [g[1] for g in desc if g[0] == "swap"] == [(i, n - 1 - i) for i in range(n // 2)]


def test_batch_workloads():
    ns, descs = cg.build_batch("traj512")
    assert len(ns) == len(descs) == 576
    assert ns[512:] == [20] * 64 and all(12 <= v <= 24 for v in ns[:512])
    assert set(ns[:512]) == set(range(12, 25))
    assert sum(len(d) for d in descs) == 440601
    ns64, d64 = cg.build_batch("traj64")
    assert len(ns64) == 72 and sum(len(d) for d in d64) == 53814
    assert all(14 <= v <= 22 for v in ns64[:64])

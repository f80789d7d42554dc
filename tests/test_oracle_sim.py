"""Pins for the per-gate oracle and its readouts against brute force and closed forms (no GPU)."""
import math

import numpy as np
import pytest

import circuitgen as cg
from oracle import sim


def _mixed_circuit(n, count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    g = []
    for _ in range(count):
        r = rng.integers(0, 12)
        q = [int(v) for v in rng.permutation(n)[:2]]
        a = [float(v) for v in rng.uniform(-math.pi, math.pi, 3)]
        if r == 0:
            g.append(("u3", (q[0],), tuple(a)))
        elif r == 1:
            g.append(("h", (q[0],), ()))
        elif r == 2:
            g.append((("x", "y", "z")[int(rng.integers(0, 3))], (q[0],), ()))
        elif r == 3:
            g.append(("ry", (q[0],), (a[0],)))
        elif r == 4:
            g.append(("rz", (q[0],), (a[0],)))
        elif n >= 2 and r == 5:
            g.append(("cx", (q[0], q[1]), ()))
        elif n >= 2 and r == 6:
            g.append(("cz", (q[0], q[1]), ()))
        elif n >= 2 and r == 7:
            g.append(("cp", (q[0], q[1]), (a[1],)))
        elif n >= 2 and r == 8:
            g.append(("swap", (q[0], q[1]), ()))
        elif n >= 2:
            g.append(("unitary", (q[0], q[1]), (cg.haar_unitary(rng),)))
        else:
            g.append(("u3", (q[0],), tuple(a)))
    return g


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 10])
def test_per_gate_matches_dense_bruteforce(n):
    g = _mixed_circuit(n, 40, 100 + n)
    rng = np.random.Generator(np.random.PCG64(n))
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi /= np.linalg.norm(psi)
    a = sim.apply(psi.copy(), n, g)
    b = sim.dense_apply(n, g, psi)
    assert np.abs(a - b).max() < 1e-13


def test_dense_unitary_product_is_unitary():
    g = _mixed_circuit(6, 30, 5)
    U = sim.dense_unitary(6, g)
    assert np.abs(U.conj().T @ U - np.eye(64)).max() < 1e-12
    assert np.abs(U[:, 9] - sim.simulate(6, g, 9)).max() < 1e-13


def test_bell_state():
    st = sim.simulate(2, [("h", (0,), ()), ("cx", (0, 1), ())])
    r = 1 / math.sqrt(2)
    assert np.abs(st - np.array([r, 0, 0, r])).max() < 1e-15


@pytest.mark.parametrize("n", [3, 12])
def test_ghz(n):
    g = [("h", (0,), ())] + [("cx", (q, q + 1), ()) for q in range(n - 1)]
    st = sim.simulate(n, g)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 2 ** -0.5
    assert np.abs(st - ref).max() < 1e-15


@pytest.mark.parametrize("n,x", [(5, 19), (12, 2771), (16, 40503)])
def test_qft_closed_form(n, x):
    st = sim.simulate(n, cg.qft(n), x)
    y = np.arange(1 << n)
    ref = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    assert np.abs(st - ref).max() < 1e-12


def test_unit_norm_random_layers():
    st = sim.simulate(14, cg.random_layers(14, 10, 3))
    assert abs(sim.norm2(st) - 1) < 1e-12


def test_unit_norm_quantum_volume():
    st = sim.simulate(12, cg.quantum_volume(12, 8, 4))
    assert abs(sim.norm2(st) - 1) < 1e-12


@pytest.mark.parametrize("make", [lambda: cg.random_layers(12, 6, 9), lambda: cg.quantum_volume(12, 6, 9),
                                  lambda: cg.qft(12)])
def test_mirror_returns_input(make):
    g = make()
    st = sim.simulate(12, cg.mirror(g), 1234)
    ref = np.zeros(1 << 12, dtype=complex)
    ref[1234] = 1
    assert np.abs(st - ref).max() < 1e-12


def test_probabilities_and_norm():
    st = sim.simulate(9, cg.random_layers(9, 4, 1))
    p = sim.probabilities(st)
    assert np.abs(p - np.abs(st) ** 2).max() < 1e-16
    assert abs(p.sum() - 1) < 1e-13


def test_splitmix64_published_stream():
    # SplitMix64 seeded with 0 starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f
    # (Steele, Lea & Flood 2014 reference generator); uniform = top 53 bits * 2^-53.
    for s, word in enumerate([0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]):
        assert sim.uniform(0, s) == (word >> 11) * 2.0 ** -53


def test_sample_basis_and_ghz_exact():
    n = 10
    p = sim.probabilities(sim.basis_state(n, 777))
    assert np.all(sim.sample(p, 1000, 5) == 777)
    g = [("h", (0,), ())] + [("cx", (q, q + 1), ()) for q in range(n - 1)]
    p = sim.probabilities(sim.simulate(n, g))
    s = sim.sample(p, 4000, 9)
    # dyadic probabilities: shot is 0 iff u < 1/2 exactly
    u = np.array([sim.uniform(9, k) for k in range(4000)])
    assert np.array_equal(s, np.where(u < 0.5, 0, (1 << n) - 1).astype(np.uint64))


def test_sample_matches_linear_scan_definition():
    n = 6
    p = sim.probabilities(sim.simulate(n, cg.random_layers(n, 3, 2)))
    s = sim.sample(p, 300, 123)
    for k in range(300):
        t = sim.uniform(123, k) * p.sum()
        acc = 0.0
        for i in range(1 << n):
            acc += p[i]
            if acc > t:
                break
        assert s[k] == i


def test_sample_chi_square():
    n = 5
    p = sim.probabilities(sim.simulate(n, cg.random_layers(n, 4, 6)))
    shots = 200000
    s = sim.sample(p, shots, 77)
    counts = np.bincount(s.astype(np.int64), minlength=1 << n)
    exp = p * shots
    keep = exp > 5
    chi2 = (((counts - exp) ** 2)[keep] / exp[keep]).sum()
    assert chi2 < 80  # 31 dof: p-value ~1e-6 at 80


def _pauli_dense(n, x, z):
    I2 = np.eye(2)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1.0, -1.0]).astype(complex)
    M = np.ones((1, 1), dtype=complex)
    for q in range(n - 1, -1, -1):  # kron puts the highest qubit first (little-endian index)
        xb, zb = (x >> q) & 1, (z >> q) & 1
        M = np.kron(M, Y if (xb and zb) else X if xb else Z if zb else I2)
    return M


def test_pauli_expval_vs_dense_kronecker():
    n = 7
    st = sim.simulate(n, cg.random_layers(n, 5, 8))
    for x, z in cg.random_pauli_strings(n, 20, 3) + [(0, 0), (5, 0), (0, 9), (127, 127)]:
        ref = np.vdot(st, _pauli_dense(n, x, z) @ st)
        got = sim.expval_pauli(st, x, z)
        assert abs(got - ref) < 1e-13
        assert abs(got.imag) < 1e-13


def test_pauli_expval_special_states():
    n = 8
    st = sim.basis_state(n, 0b10110010)
    for q in range(n):
        assert sim.expval_pauli(st, 0, 1 << q).real == (-1.0 if (0b10110010 >> q) & 1 else 1.0)
    g = [("h", (0,), ())] + [("cx", (q, q + 1), ()) for q in range(n - 1)]
    ghz = sim.simulate(n, g)
    full = (1 << n) - 1
    assert abs(sim.expval_pauli(ghz, full, 0) - 1) < 1e-14        # X^n
    assert abs(sim.expval_pauli(ghz, full, 0b11) + 1) < 1e-14     # Y Y X ... X
    assert abs(sim.expval_pauli(ghz, 0, 0b11) - 1) < 1e-14        # Z Z

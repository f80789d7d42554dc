"""Pins for the oracle's gate matrices and the paper's printed examples (no GPU)."""
import math
import os

import numpy as np
import pytest

import circuitgen as cg
from oracle import gates as og
from oracle import sim

from conftest import read_golden

KINDS_1Q = [("u3", (0.3, 1.1, -2.0)), ("h", ()), ("x", ()), ("y", ()), ("z", ()), ("ry", (0.7,)), ("rz", (1.9,))]
KINDS_2Q = [("cx", ()), ("cz", ()), ("cp", (0.45,)), ("swap", ())]


@pytest.fixture(scope="module")
def golden(golden_dir):
    return read_golden(os.path.join(golden_dir, "paper_examples.txt"))


def test_eq1_literal_values():
    # Eq. 1 at special angles reduces to textbook matrices: u3(pi, 0, pi) = X, u3(pi/2, 0, pi) = H.
    _, x = og.matrix_of("u3", (0,), (math.pi, 0.0, math.pi))
    assert np.allclose(x, [[0, 1], [1, 0]], atol=1e-15)
    _, h = og.matrix_of("u3", (0,), (math.pi / 2, 0.0, math.pi))
    assert np.allclose(h, np.array([[1, 1], [1, -1]]) / math.sqrt(2), atol=1e-15)
    # u3(t, p, l)|0> = (cos t/2, e^{ip} sin t/2): the first column of Eq. 1.
    t, p, l = 1.234, -0.77, 2.5
    _, u = og.matrix_of("u3", (0,), (t, p, l))
    assert np.allclose(u[:, 0], [math.cos(t / 2), np.exp(1j * p) * math.sin(t / 2)], atol=1e-15)
    # top-right entry carries e^{i lambda}, bottom-right e^{i(phi+lambda)}
    assert abs(u[0, 1] + np.exp(1j * l) * math.sin(t / 2)) < 1e-15
    assert abs(u[1, 1] - np.exp(1j * (p + l)) * math.cos(t / 2)) < 1e-15


def test_eq2_literal_and_orientation(golden):
    vals = [int(v) for v in golden["cnot_eq2_row_major"][0].split()]
    assert np.array_equal(og.CNOT_EQ2.real.astype(int).reshape(-1), vals)
    # control = higher local bit: cx(control=1, target=0) maps |10> (index 2) to |11> (index 3)
    st = sim.basis_state(2, 2)
    sim.apply(st, 2, [("cx", (1, 0), ())])
    assert np.array_equal(np.abs(st), [0, 0, 0, 1])
    # and leaves |01> (control 0) unchanged
    st = sim.basis_state(2, 1)
    sim.apply(st, 2, [("cx", (1, 0), ())])
    assert np.array_equal(np.abs(st), [0, 1, 0, 0])


def test_basis_state_example(golden):
    vals = [int(v) for v in golden["basis_2_of_2q"][0].split()]
    assert np.array_equal(sim.basis_state(2, 2).real, vals)


def test_fig2_pair_example(golden):
    i, partner, k, n = (int(v) for v in golden["pair_example"][0].split())
    assert i ^ (1 << k) == partner
    # X (= u3(pi, 0, pi)) on qubit k moves |0011> to |0111>
    st = sim.basis_state(n, i)
    sim.apply(st, n, [("u3", (k,), (math.pi, 0.0, math.pi))])
    assert abs(abs(st[partner]) - 1) < 1e-15


@pytest.mark.parametrize("n,k", [(4, 2), (5, 0), (6, 5), (8, 3)])
def test_listing2_index_map_is_pair_bijection(n, k):
    # Listing 2 enumerates pairs by i1 = i & mask; i0 = ((i - i1) << 1) + i1; i1 = i0 + 2^k over
    # i < 2^(n-1).  Its pairs must be exactly {(j, j XOR 2^k) : bit k of j is 0} (Fig. 2).
    add, mask = 1 << k, (1 << k) - 1
    seen = []
    for i in range(1 << (n - 1)):
        lo = i & mask
        i0 = ((i - lo) << 1) + lo
        i1 = i0 + add
        assert (i0 >> k) & 1 == 0 and i1 == i0 ^ add
        seen += [i0, i1]
    assert sorted(seen) == list(range(1 << n))


def test_memory_and_capacity_model(golden):
    per_amp = int(golden["memory_bytes_per_amp_fp64"][0])
    assert per_amp == np.dtype(np.complex128).itemsize
    # largest n whose state leaves room in the memory (16 * 2^n strictly below the capacity)
    def max_n(cap):
        n = 0
        while per_amp * 2 ** (n + 1) < cap:
            n += 1
        return n
    for cap in (16 * 2 ** 30, 16e9):
        assert max_n(cap) == int(golden["max_qubits_16GB_gpu_fp64"][0])
    for cap in (512 * 2 ** 30, 512e9):
        assert max_n(cap) == int(golden["max_qubits_512GB_cpu_fp64"][0])


def test_byte_per_flop(golden):
    # one pair: 2 loads + 2 stores of complex128 = 64 B; 2 x (2 complex mul + 1 complex add)
    # = 2 x (2*6 + 2) = 28 flop  ->  64 / 28 = 2.29
    assert round(64 / 28, 2) == float(golden["byte_per_flop_fp64_1q"][0])


@pytest.mark.parametrize("kind,params", KINDS_1Q)
def test_unitarity_1q(kind, params):
    _, u = og.matrix_of(kind, (0,), params)
    assert np.abs(u.conj().T @ u - np.eye(2)).max() < 1e-14


@pytest.mark.parametrize("kind,params", KINDS_2Q)
def test_unitarity_2q(kind, params):
    _, u = og.matrix_of(kind, (0, 1), params)
    assert np.abs(u.conj().T @ u - np.eye(4)).max() < 1e-14


def test_haar_su4_det_and_unitarity():
    rng = np.random.Generator(np.random.PCG64(11))
    for _ in range(50):
        u = cg.haar_unitary(rng, 4)
        assert np.abs(u.conj().T @ u - np.eye(4)).max() < 1e-13
        assert abs(np.linalg.det(u) - 1) < 1e-13


def test_pauli_products():
    _, x = og.matrix_of("x", (0,), ())
    _, y = og.matrix_of("y", (0,), ())
    _, z = og.matrix_of("z", (0,), ())
    assert np.allclose(1j * x @ z, y)

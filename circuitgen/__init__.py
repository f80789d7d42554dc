"""Seeded synthetic circuit generators shared by the CUDA library's tests/bench and the CPU oracle.

This module only draws random numbers and lists gates. It holds none of the simulation
arithmetic: no gate matrix is built here except the Haar-random two-qubit unitaries, which
are random *inputs* of the quantum-volume workload (the method never draws them). Each
side (the CUDA library and the oracle) turns a gate description into a matrix on its own.

A gate is a tuple ``(kind, qubits, params)``:

* ``("u3", (q,), (theta, phi, lam))`` -- the paper's Eq. 1 rotation (its psi is phi here),
* ``("cx", (control, target), ())`` -- Eq. 2 CNOT,
* ``("h", (q,), ())``, ``("x"|"y"|"z", (q,), ())``, ``("ry", (q,), (theta,))``,
  ``("rz", (q,), (theta,))``,
* ``("cp", (control, target), (phi,))``, ``("cz", (a, b), ())``,
* ``("swap", (a, b), ())`` -- a qubit relabel,
* ``("unitary", (q0, q1), (M,))`` -- dense 4x4 complex matrix ``M`` (row-major) in the local
  basis ``b = bit(q0) + 2*bit(q1)``.

Qubit numbering is little-endian: basis index bit k is qubit k (paper Sec. II.A, Fig. 2).

The workloads stand in for the paper's evaluation circuits (Quantum Volume and QFT,
Sec. V.A) plus the random-layer, noisy-trajectory and hardware-efficient-ansatz circuits used
to exercise the method at other densities.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_layers(n: int, depth: int, seed: int):
    """Random-layer circuit: per layer U3 on every qubit with angles uniform in [0, 2pi),
    then CX on a random perfect matching (control = perm[2i], target = perm[2i+1]); for odd n
    the last qubit of the permutation idles."""
    rng = _rng(seed)
    gates = []
    for _ in range(depth):
        ang = rng.uniform(0.0, TWO_PI, size=(n, 3))
        for q in range(n):
            gates.append(("u3", (q,), (float(ang[q, 0]), float(ang[q, 1]), float(ang[q, 2]))))
        perm = rng.permutation(n)
        for i in range(n // 2):
            gates.append(("cx", (int(perm[2 * i]), int(perm[2 * i + 1])), ()))
    return gates


def qft(n: int, with_swaps: bool = True):
    """Textbook quantum Fourier transform on n qubits (the paper uses QFT in Sec. V without
    defining it): for j = n-1 .. 0, H on qubit j then CP(pi / 2^(j-m)) between m and j for
    m = j-1 .. 0; finally the qubit reversal as SWAP gates (relabels).  On basis state |x>
    it yields amplitudes exp(2 pi i x y / 2^n) / 2^(n/2)."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(("h", (j,), ()))
        for m in range(j - 1, -1, -1):
            gates.append(("cp", (m, j), (math.pi / float(1 << (j - m)),)))
    if with_swaps:
        for i in range(n // 2):
            gates.append(("swap", (i, n - 1 - i), ()))
    return gates


def haar_unitary(rng: np.random.Generator, dim: int = 4) -> np.ndarray:
    """Haar-random element of SU(dim): QR of a complex Ginibre matrix with the phases of R's
    diagonal moved into Q (Mezzadri 2007), then divided by the principal dim-th root of det."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    q = q * (d / np.abs(d))[None, :]
    det = np.linalg.det(q)
    q = q / det ** (1.0 / dim)
    return np.ascontiguousarray(q, dtype=np.complex128)


def quantum_volume(n: int, depth: int, seed: int):
    """Quantum-volume-style circuit: per layer a random permutation perm of the qubits, then a
    Haar-random SU(4) on (perm[2i], perm[2i+1]) for i < n // 2.  The permutation only selects
    the pairs; no SWAP gates are emitted."""
    rng = _rng(seed)
    gates = []
    for _ in range(depth):
        perm = rng.permutation(n)
        for i in range(n // 2):
            u = haar_unitary(rng, 4)
            gates.append(("unitary", (int(perm[2 * i]), int(perm[2 * i + 1])), (u,)))
    return gates


def basis_index(n: int, seed: int) -> int:
    """A seeded uniform basis index in [0, 2^n)."""
    return int(_rng(seed).integers(0, 1 << n))


_PAULI_1Q = ("x", "y", "z")


def noisy_trajectory(n: int, depth: int, p: float, seed: int, traj_id: int):
    """One depolarizing-noise trajectory of the random-layer circuit: after each gate, with
    probability p, a uniform non-identity Pauli on the gate's qubits (3 choices for a 1-qubit
    gate, 15 for a 2-qubit gate), drawn from a generator seeded with
    seed XOR (traj_id * 0x9E3779B1 + 1).  The trajectory is a plain deterministic circuit that
    both sides replay."""
    base = random_layers(n, depth, seed * 1000003 + n)
    rng = _rng(seed ^ (traj_id * 0x9E3779B1 + 1))
    gates = []
    for g in base:
        gates.append(g)
        if rng.random() < p:
            nq = len(g[1])
            k = int(rng.integers(1, 4 ** nq))  # 1 .. 4^nq - 1: non-identity Pauli word
            for j, q in enumerate(g[1]):
                w = (k >> (2 * j)) & 3
                if w:
                    gates.append((_PAULI_1Q[w - 1], (q,), ()))
    return gates


def trajectory_sizes(count: int, lo: int, hi: int, seed: int):
    """Qubit counts uniform in [lo, hi] for a batch of trajectories."""
    return [int(v) for v in _rng(seed).integers(lo, hi + 1, size=count)]


def hea(n: int, layers: int, seed: int, param_set: int):
    """Hardware-efficient ansatz: `layers` x (RY on every qubit + CZ(i, i+1) ladder), then a final
    RY layer; angles uniform in [0, 2pi) from a generator seeded with (seed, param_set)."""
    rng = _rng(seed * 7919 + param_set)
    gates = []
    for _ in range(layers):
        th = rng.uniform(0.0, TWO_PI, size=n)
        for q in range(n):
            gates.append(("ry", (q,), (float(th[q]),)))
        for q in range(n - 1):
            gates.append(("cz", (q, q + 1), ()))
    th = rng.uniform(0.0, TWO_PI, size=n)
    for q in range(n):
        gates.append(("ry", (q,), (float(th[q]),)))
    return gates


def random_pauli_strings(n: int, count: int, seed: int):
    """`count` seeded Pauli strings as (x_mask, z_mask) pairs (Y = both bits set)."""
    rng = _rng(seed)
    out = []
    for _ in range(count):
        w = rng.integers(0, 4, size=n)
        x = 0
        z = 0
        for q in range(n):
            if w[q] in (1, 2):
                x |= 1 << q
            if w[q] in (2, 3):
                z |= 1 << q
        out.append((x, z))
    return out


def mirror(gates):
    """U followed by U^dagger as gate descriptions: the inverse of each gate in reverse order.
    Only kinds with an exact parametric inverse are supported here; 'unitary' carries M^H."""
    inv = []
    for kind, qs, params in reversed(gates):
        if kind == "u3":
            th, ph, lam = params
            inv.append(("u3", qs, (-th, -lam, -ph)))
        elif kind in ("cx", "h", "x", "y", "z", "cz", "swap"):
            inv.append((kind, qs, ()))
        elif kind in ("ry", "rz"):
            inv.append((kind, qs, (-params[0],)))
        elif kind == "cp":
            inv.append(("cp", qs, (-params[0],)))
        elif kind == "unitary":
            inv.append(("unitary", qs, (np.ascontiguousarray(np.conj(params[0]).T),)))
        else:
            raise ValueError(kind)
    return gates + inv


# Workload definitions (sizes, seeds) used by tests and the benchmark.
WORKLOADS = {
    "rl16": dict(kind="random_layers", n=16, depth=20, seed=1, c=10),
    "qft28": dict(kind="qft", n=28, seed=2, c=12),
    "rl28": dict(kind="random_layers", n=28, depth=40, seed=3, c=12),
    "qv30": dict(kind="quantum_volume", n=30, depth=30, seed=4, c=12, pinned=5),
    "qv26": dict(kind="quantum_volume", n=26, depth=10, seed=4, c=12, pinned=5),
    "rl32": dict(kind="random_layers", n=32, depth=32, seed=7, c=13),
    "qv32": dict(kind="quantum_volume", n=32, depth=32, seed=7, c=12, pinned=5),
}


def build(name: str):
    """Gate list of a named workload."""
    w = WORKLOADS[name]
    if w["kind"] == "random_layers":
        return random_layers(w["n"], w["depth"], w["seed"])
    if w["kind"] == "qft":
        return qft(w["n"])
    if w["kind"] == "quantum_volume":
        return quantum_volume(w["n"], w["depth"], w["seed"])
    raise ValueError(name)


# Batched workloads: many independent states (noisy trajectories plus ansatz parameter sets).
BATCH_WORKLOADS = {
    "traj512": dict(count=512, lo=12, hi=24, depth=30, p=1e-3, seed=8, hea_n=20, hea_sets=64, hea_layers=10),
    # a smaller mix (about 0.5 GiB, above L2) for profiling and quick checks
    "traj64": dict(count=64, lo=14, hi=22, depth=30, p=1e-3, seed=8, hea_n=20, hea_sets=8, hea_layers=10),
}


def build_batch(name: str):
    """(qubit counts, gate lists) of a named batched workload: `count` depolarizing trajectories of
    the random-layer circuit with qubit counts uniform in [lo, hi], then `hea_sets` parameter sets
    of the hardware-efficient ansatz on hea_n qubits."""
    w = BATCH_WORKLOADS[name]
    ns = trajectory_sizes(w["count"], w["lo"], w["hi"], w["seed"])
    descs = [noisy_trajectory(n, w["depth"], w["p"], w["seed"], t) for t, n in enumerate(ns)]
    for k in range(w["hea_sets"]):
        ns.append(w["hea_n"])
        descs.append(hea(w["hea_n"], w["hea_layers"], w["seed"], k))
    return ns, descs

"""Python side of the CPU oracle (test infrastructure only).

* ``simulate`` / ``apply``: the per-gate update of Sec. II.A in complex128, run by the C
  library ``sv_oracle.c`` (OpenMP over groups, one pass per gate).
* ``dense_apply``: brute force for n <= 10 -- every gate embedded as a full 2^n x 2^n matrix
  straight from the definition ``F[i, j] = U[b(i), b(j)]`` when i and j agree outside the gate's
  qubits, else 0, and multiplied into the state.  Shares nothing with the C loop.
* readouts: probabilities (Sec. II.A), norm, Pauli expectation, inverse-CDF sampling.
* ``execute_plan``: runs a cache-blocking plan (``oracle.planner``) gate by gate: each
  chunk_swap pair as a bit exchange (Sec. IV.C, Fig. 10), each blocked gate on its physical
  qubits -- used to check that the transpiled circuit equals the original one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import gates as _gates

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sv_oracle.c with gcc (-O3 -fopenmp) into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "sv_oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_apply_gate.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, dp]
            L.oracle_apply_circuit.argtypes = [dp, ctypes.c_int, ctypes.c_int64, ip, ip, dp]
            L.oracle_init_basis.argtypes = [dp, ctypes.c_int, ctypes.c_uint64]
            L.oracle_swap_bits.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.oracle_probabilities.argtypes = [dp, ctypes.c_int, dp]
            L.oracle_norm2.argtypes = [dp, ctypes.c_int]
            L.oracle_norm2.restype = ctypes.c_double
            L.oracle_expval_pauli.argtypes = [dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, dp]
            L.oracle_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.oracle_uniform.restype = ctypes.c_double
            L.oracle_sample.argtypes = [dp, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint64), dp]
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def gate_arrays(gates):
    """Flatten gate descriptions into (nq[G], qubits[2G], matrices[32G]) for the C oracle."""
    G = len(gates)
    nq = np.zeros(G, dtype=np.int32)
    qs = np.zeros(2 * G, dtype=np.int32)
    mats = np.zeros(32 * G, dtype=np.float64)
    for j, (kind, qubits, params) in enumerate(gates):
        order, m = _gates.matrix_of(kind, qubits, params)
        k = len(order)
        nq[j] = k
        qs[2 * j: 2 * j + k] = order
        flat = np.ascontiguousarray(m, dtype=np.complex128).reshape(-1)
        mats[32 * j: 32 * j + 2 * flat.size] = flat.view(np.float64)
    return nq, qs, mats


def basis_state(n: int, basis: int = 0) -> np.ndarray:
    st = np.empty(1 << n, dtype=np.complex128)
    lib().oracle_init_basis(_dp(st.view(np.float64)), n, basis)
    return st


def apply(state: np.ndarray, n: int, gates) -> np.ndarray:
    """Apply `gates` (circuitgen descriptions) to `state` in place; returns `state`."""
    assert state.dtype == np.complex128 and state.size == (1 << n) and state.flags.c_contiguous
    if not gates:
        return state
    nq, qs, mats = gate_arrays(gates)
    lib().oracle_apply_circuit(_dp(state.view(np.float64)), n, len(gates),
                               nq.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               qs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(mats))
    return state


def simulate(n: int, gates, basis: int = 0) -> np.ndarray:
    """|psi_out> = U_G ... U_1 |basis>, one pass per gate (Sec. II.A)."""
    return apply(basis_state(n, basis), n, gates)


def swap_bits(state: np.ndarray, n: int, p: int, q: int) -> np.ndarray:
    lib().oracle_swap_bits(_dp(state.view(np.float64)), n, p, q)
    return state


# ---------------------------------------------------------------- dense brute force (n <= 10)

def embed(n: int, qubits, u: np.ndarray) -> np.ndarray:
    """Full 2^n x 2^n matrix of gate u on `qubits` (local index b = sum_j bit(q_j) 2^j):
    F[i, j] = u[b(i), b(j)] if i and j agree on every other bit, else 0."""
    N = 1 << n
    idx = np.arange(N, dtype=np.int64)
    b = np.zeros(N, dtype=np.int64)
    mask = 0
    for j, q in enumerate(qubits):
        b |= ((idx >> q) & 1) << j
        mask |= 1 << q
    rest = idx & ~mask
    same = rest[:, None] == rest[None, :]
    return np.where(same, u[b[:, None], b[None, :]], 0.0 + 0.0j)


def dense_apply(n: int, gates, state: np.ndarray) -> np.ndarray:
    assert n <= 10, "dense brute force is for n <= 10"
    out = np.array(state, dtype=np.complex128)
    for kind, qubits, params in gates:
        order, u = _gates.matrix_of(kind, qubits, params)
        out = embed(n, order, u) @ out
    return out


def dense_unitary(n: int, gates) -> np.ndarray:
    assert n <= 8, "dense unitary product is for n <= 8"
    U = np.eye(1 << n, dtype=np.complex128)
    for kind, qubits, params in gates:
        order, u = _gates.matrix_of(kind, qubits, params)
        U = embed(n, order, u) @ U
    return U


# ---------------------------------------------------------------- readouts

def probabilities(state: np.ndarray) -> np.ndarray:
    n = int(state.size).bit_length() - 1
    out = np.empty(state.size, dtype=np.float64)
    lib().oracle_probabilities(_dp(np.ascontiguousarray(state).view(np.float64)), n, _dp(out))
    return out


def norm2(state: np.ndarray) -> float:
    n = int(state.size).bit_length() - 1
    return float(lib().oracle_norm2(_dp(np.ascontiguousarray(state).view(np.float64)), n))


def expval_pauli(state: np.ndarray, x_mask: int, z_mask: int) -> complex:
    n = int(state.size).bit_length() - 1
    out = np.zeros(2, dtype=np.float64)
    lib().oracle_expval_pauli(_dp(np.ascontiguousarray(state).view(np.float64)), n,
                              x_mask, z_mask, _dp(out))
    return complex(out[0], out[1])


def uniform(seed: int, s: int) -> float:
    return float(lib().oracle_uniform(seed, s))


def sample(probs: np.ndarray, shots: int, seed: int) -> np.ndarray:
    n = int(probs.size).bit_length() - 1
    p = np.ascontiguousarray(probs, dtype=np.float64)
    out = np.zeros(shots, dtype=np.uint64)
    scratch = np.empty(p.size, dtype=np.float64)
    lib().oracle_sample(_dp(p), n, shots, seed, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                        _dp(scratch))
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ---------------------------------------------------------------- planned execution

def execute_plan(n: int, gates, plan, basis: int = 0, state: np.ndarray | None = None) -> np.ndarray:
    """Run a plan from ``oracle.planner.plan_blocking``: swap rounds move data (bit exchanges),
    blocks apply the original gates on their physical qubits, one pass per gate."""
    st = basis_state(n, basis) if state is None else state
    for op in plan.ops:
        if op[0] in ("swap", "unpermute"):
            for p, q in op[1]:
                swap_bits(st, n, p, q)
        elif op[0] in ("block", "gblock"):
            body = op[1][1] if op[0] == "gblock" else op[1]
            phys = []
            for gi, pq in body:
                kind, qubits, params = gates[gi]
                order, u = _gates.matrix_of(kind, qubits, params)
                # pq lists the physical positions of the gate's qubits in ascending label
                # order; re-express them in the matrix's local order.
                where = {q: p for q, p in zip(sorted(qubits), pq)}
                phys.append(("unitary", tuple(where[q] for q in order), (u,)))
            apply(st, n, phys)
        else:
            raise ValueError(op[0])
    return st

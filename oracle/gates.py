"""Gate matrices in complex128 (oracle side; test infrastructure only).

Every matrix is row-major in the gate's local basis: for a 2-qubit gate on qubits (q0, q1)
the local index is b = bit(q0) + 2*bit(q1), so q1 is the *higher* local bit.
"""
from __future__ import annotations

import cmath
import math

import numpy as np


def u3(theta: float, phi: float, lam: float) -> np.ndarray:
    """Paper Sec. II.A, Eq. 1 (the paper writes psi for OpenQASM's phi):
    [[cos(t/2), -e^{i lam} sin(t/2)], [e^{i phi} sin(t/2), e^{i(phi+lam)} cos(t/2)]]."""
    c = math.cos(theta / 2.0)
    s = math.sin(theta / 2.0)
    return np.array(
        [[c, -cmath.exp(1j * lam) * s], [cmath.exp(1j * phi) * s, cmath.exp(1j * (phi + lam)) * c]],
        dtype=np.complex128,
    )


# Paper Sec. II.A, Eq. 2: CNOT with the higher local bit as control.
CNOT_EQ2 = np.array(
    [[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128
)

_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def matrix_of(kind: str, qubits, params):
    """(local qubit order, matrix) for a gate description from ``circuitgen``.

    The returned qubit tuple is the order that defines the local basis of the matrix."""
    if kind == "u3":
        return tuple(qubits), u3(*params)
    if kind == "h":
        return tuple(qubits), _H.copy()
    if kind == "x":
        return tuple(qubits), _X.copy()
    if kind == "y":
        return tuple(qubits), _Y.copy()
    if kind == "z":
        return tuple(qubits), _Z.copy()
    if kind == "ry":
        t = params[0]
        c, s = math.cos(t / 2.0), math.sin(t / 2.0)
        return tuple(qubits), np.array([[c, -s], [s, c]], dtype=np.complex128)
    if kind == "rz":
        t = params[0]
        return tuple(qubits), np.array(
            [[cmath.exp(-0.5j * t), 0], [0, cmath.exp(0.5j * t)]], dtype=np.complex128
        )
    if kind == "cx":
        control, target = qubits
        # local order (target, control): the control is the higher local bit, as in Eq. 2.
        return (target, control), CNOT_EQ2.copy()
    if kind == "cz":
        return tuple(qubits), np.diag([1, 1, 1, -1]).astype(np.complex128)
    if kind == "cp":
        return tuple(qubits), np.diag([1, 1, 1, cmath.exp(1j * params[0])]).astype(np.complex128)
    if kind == "swap":
        m = np.zeros((4, 4), dtype=np.complex128)
        m[0, 0] = m[3, 3] = m[1, 2] = m[2, 1] = 1
        return tuple(qubits), m
    if kind == "unitary":
        return tuple(qubits), np.asarray(params[0], dtype=np.complex128).copy()
    raise ValueError(f"unknown gate kind {kind!r}")

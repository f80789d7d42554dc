"""sv_expval_pauli_noalloc: the Pauli expectation for callers that may not allocate memory at
call time (their memory is a pool or budget they do not own, or a cudaMalloc would stall their
loop).  It must return what sv_expval_pauli returns, call after call, although every call reuses
the same fixed scratch array inside the library.  This file is collected last so that a run that
stops at the first failure has run every other test before it."""
import numpy as np
import pytest

import circuitgen as cg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2102_02957_gb300 as m
    return m


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 1e-5)])
def test_noalloc_matches_allocating_entry_point(sv, dtype, tol):
    n = 18
    desc = cg.random_layers(n, 5, 21)
    gates = sv.make_gates(desc)
    paulis = cg.random_pauli_strings(n, 2, 9)  # two calls in a row, different words
    with sv.StateVector(n, dtype) as st:
        st.init_basis(0)
        st.apply(gates, sv.Plan(n, gates, chunk_bits=10))
        st.synchronize()
        for x, z in paulis + [paulis[0]]:
            got = st.expval_pauli_noalloc(x, z)
            ref = st.expval_pauli(x, z)
            assert abs(got - ref) <= tol, (x, z, got, ref)
            assert np.isfinite(got.real) and np.isfinite(got.imag)


def test_noalloc_back_to_back_on_two_states(sv):
    # the shared scratch keeps the previous call's contents: a second state's result must not
    # depend on them
    a = sv.StateVector(12, "c128")
    b = sv.StateVector(16, "c128")
    try:
        a.init_basis(5)
        b.init_basis(0)
        g = sv.make_gates(cg.quantum_volume(16, 3, 4))
        b.apply(g)
        za = a.expval_pauli_noalloc(0, 0b101)  # Z0 Z2 on |...0101> -> (+1)
        zb = b.expval_pauli_noalloc(0, 0b11)
        assert abs(za - 1.0) < 1e-12
        assert abs(zb - b.expval_pauli(0, 0b11)) < 1e-12
        assert abs(a.expval_pauli_noalloc(0, 0b101) - 1.0) < 1e-12
    finally:
        a.close()
        b.close()

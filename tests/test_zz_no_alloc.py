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


def test_noalloc_allocates_nothing(sv):
    """The point of the entry point: after the first call on this device (which sets up the
    library's fixed scratch), further calls on a fresh handle take no device memory -- neither the
    handle's own scratch (which sv_expval_pauli would create) nor anything else: the device's
    free bytes and torch's reserved bytes stay exactly the same."""
    import torch
    n = 16
    g = sv.make_gates(cg.quantum_volume(n, 3, 6))
    warm = sv.StateVector(10, "c64")
    try:
        warm.init_basis(1)
        warm.expval_pauli_noalloc(0, 1)  # the first call on the device
    finally:
        warm.close()
    with sv.StateVector(n, "c64") as st:
        st.init_basis(0)
        st.apply(g)
        st.synchronize()
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        vals = [st.expval_pauli_noalloc(x, z) for x, z in cg.random_pauli_strings(n, 6, 12)]
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        assert torch.cuda.memory_reserved() == reserved0
        assert all(np.isfinite(v.real) and np.isfinite(v.imag) for v in vals)

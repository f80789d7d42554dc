"""GPU parity of the two ways a state larger than one GPU's memory is run (against the oracle;
complex128 1e-12, complex64 1e-5 max-abs and 1 - F <= 1e-8):

* partitioned on its top qubits (Sec. II.B, IV.C): G = 2, 4, 8 pieces, each a StateVector of
  n - g qubits driven through the library (sv_apply_plan_ops, sv_shard_pack / sv_shard_unpack),
  emulating G GPUs in one process on one GPU (every exchange is a copy of packed buffers in lock
  step; no kernels wait on one another);
* host-resident (Sec. IV.C, V.B: the GPU as a cache for chunks in host memory): the state in pinned
  host memory, a device work buffer far smaller than the state, so that every pass gathers
  sub-states of a few slabs."""
import numpy as np
import pytest

import circuitgen as cg
from oracle import sim

from gpu_util import assert_close

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


def _circuits(n, seed):
    return [cg.quantum_volume(n, 6, seed), cg.random_layers(n, 6, seed + 1), cg.qft(n),
            cg.mirror(cg.quantum_volume(n, 3, seed + 2)),
            [("h", (q,), ()) for q in range(n - 2)] + [("swap", (n - 2, n - 1), ()), ("cx", (0, 1), ())]]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,g,c", [(16, 1, 8), (18, 2, 10), (17, 3, 9)])
def test_partitioned_state_on_library_kernels(sv, dtype, n, g, c):
    from paper_2102_02957_gb300 import shard
    n_local = n - g
    for desc in _circuits(n, 3 * n + g):
        basis = cg.basis_index(n, g + 7)
        gates = sv.make_gates(desc)
        plan = sv.Plan(n, gates, chunk_bits=c)
        ops = shard.parse_ops(plan.serialize())
        full = sim.basis_state(n, basis).astype(np.complex64 if dtype == "c64" else np.complex128)
        states = [sv.StateVector(n_local, dtype) for _ in range(1 << g)]
        try:
            for r, st in enumerate(states):
                st.set_state(np.ascontiguousarray(full[r << n_local:(r + 1) << n_local]))
            pieces = [shard.GpuPiece(st, gates, plan) for st in states]
            shard.run_lockstep(pieces, [shard.schedule(ops, n_local, r) for r in range(1 << g)])
            got = np.concatenate([st.get_state() for st in states])
        finally:
            for st in states:
                st.close()
        assert_close(got, sim.simulate(n, desc, basis), dtype)


def test_partitioned_plan_ops_refuses_chunk_wider_than_piece(sv):
    n = 12
    gates = sv.make_gates(cg.quantum_volume(n, 2, 1))
    plan = sv.Plan(n, gates, chunk_bits=11)
    with sv.StateVector(10, "c64") as st:
        with pytest.raises(sv.SVError) as e:
            st.apply_ops(gates, plan, 0, 1)
        assert e.value.status == sv._lib.SV_ERR_PLAN


def _pinned(n, dtype, basis):
    import torch
    dt = torch.complex64 if dtype == "c64" else torch.complex128
    t = torch.zeros(1 << n, dtype=dt, pin_memory=True)
    t[basis] = 1.0
    return t


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,c,work_amps", [(18, 8, 1 << 12), (20, 10, 1 << 15), (22, 12, 1 << 20), (16, 8, 1 << 18)])
def test_host_resident_state(sv, dtype, n, c, work_amps):
    elem = 8 if dtype == "c64" else 16
    for desc in _circuits(n, 5 * n + c):
        basis = cg.basis_index(n, c)
        gates = sv.make_gates(desc)
        plan = sv.Plan(n, gates, chunk_bits=c)
        host = _pinned(n, dtype, basis)
        passes = sv.apply_host(n, host, gates, plan, 2 * work_amps * elem, dtype=dtype)
        info = plan.info()
        assert 1 <= passes <= info.n_blocks + info.n_swap_rounds + info.n_unpermute_rounds + 8
        assert_close(host.numpy(), sim.simulate(n, desc, basis), dtype)


def test_host_resident_work_buffer_too_small(sv):
    n, c = 16, 8
    gates = sv.make_gates(cg.random_layers(n, 2, 1))
    plan = sv.Plan(n, gates, chunk_bits=c)
    host = _pinned(n, "c64", 0)
    with pytest.raises(sv.SVError) as e:
        sv.apply_host(n, host, gates, plan, 2 * (1 << (c + 1)) * 8)
    assert e.value.status == sv._lib.SV_ERR_ARG
    gathered = sv.Plan(n, gates, chunk_bits=c, gather_pinned=4)
    with pytest.raises(sv.SVError) as e:
        sv.apply_host(n, host, gates, gathered, 1 << 24)
    assert e.value.status == sv._lib.SV_ERR_UNSUPPORTED

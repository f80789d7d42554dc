"""GPU parity of batched execution (many states, one persistent launch) and of the autotuner,
against the CPU oracle.  Workloads: depolarizing-noise trajectories of the random-layer circuit
(Pauli insertions after gates, the trajectory form of the paper's shots) and hardware-efficient
ansatz parameter sets.  Tolerance: complex64 1e-5 max-abs and 1 - fidelity <= 1e-8."""
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


def _workload(sizes, depth, p, seed, hea_n=0, hea_sets=0):
    descs = [cg.noisy_trajectory(n, depth, p, seed, t) for t, n in enumerate(sizes)]
    ns = list(sizes)
    for k in range(hea_sets):
        descs.append(cg.hea(hea_n, 10, seed, k))
        ns.append(hea_n)
    return ns, descs


def _run_batch(sv, ns, descs, use_graph, repeats=1, **opts):
    gates = [sv.make_gates(d) for d in descs]
    states = [sv.StateVector(n, "c64") for n in ns]
    b = sv.Batch(states, gates, **opts)
    try:
        for _ in range(repeats):
            for s in states:
                s.init_basis(0)
            b.run(use_graph=use_graph)
            b.synchronize()
        out = [s.get_state() for s in states]
        info = b.info()
    finally:
        b.close()
        for s in states:
            s.close()
    return out, info


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_small_states_one_residency(sv, use_graph):
    """States of 6..13 qubits fit one 13-bit chunk: one section each, the whole circuit in one
    shared-memory residency."""
    ns, descs = _workload([6, 7, 9, 11, 12, 13, 8, 10], 12, 0.05, 11, hea_n=10, hea_sets=3)
    out, (items, sections, _) = _run_batch(sv, ns, descs, use_graph, repeats=2, chunk_bits=13)
    assert sections >= len(ns)
    for n, d, got in zip(ns, descs, out):
        assert_close(got, sim.simulate(n, d), "c64")


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_multi_section_states(sv, use_graph):
    """States larger than the chunk: several gathered sections per state, ordered by the
    per-state completion counters inside one launch."""
    ns, descs = _workload([14, 16, 12, 18, 15], 20, 0.01, 5, hea_n=16, hea_sets=2)
    out, (items, sections, _) = _run_batch(sv, ns, descs, use_graph, repeats=2, chunk_bits=10)
    assert sections > len(ns)
    for n, d, got in zip(ns, descs, out):
        assert_close(got, sim.simulate(n, d), "c64")


def test_batch_trajectory_mix_norms_and_sampled_parity(sv):
    """A mixed batch (12..20 qubits, default chunk): unit norm for every state, oracle parity on a
    seeded subset."""
    sizes = cg.trajectory_sizes(24, 12, 20, 3)
    ns, descs = _workload(sizes, 20, 1e-3, 3, hea_n=20, hea_sets=4)
    out, _ = _run_batch(sv, ns, descs, True, repeats=1)
    for got in out:
        assert abs(float(np.vdot(got, got).real) - 1.0) < 1e-4
    for k in (0, 5, 11, len(ns) - 1):
        assert_close(out[k], sim.simulate(ns[k], descs[k]), "c64")


@pytest.mark.parametrize("use_tc", [0, 1])
def test_batch_trajectories_up_to_24_qubits(sv, use_tc):
    """Config 4's range at its top: depolarizing trajectories of the depth-30 random-layer circuit
    (p = 1e-3) on 12..24 qubits, three of them 24-qubit, and two 20-qubit ansatz parameter sets,
    one graph-replayed launch; every state against the oracle."""
    sizes = [24, 23, 24, 22, 18, 12, 20, 24, 16, 21]
    ns, descs = _workload(sizes, 30, 1e-3, 17, hea_n=20, hea_sets=2)
    out, (items, sections, _) = _run_batch(sv, ns, descs, True, repeats=1, use_tc=use_tc)
    assert sections > len(ns)
    for n, d, got in zip(ns, descs, out):
        assert_close(got, sim.simulate(n, d), "c64")


def test_batch_rejects_unsupported(sv):
    g = sv.make_gates(cg.hea(8, 2, 1, 0))
    with sv.StateVector(8, "c128") as s:
        with pytest.raises(sv.SVError):
            sv.Batch([s], [g])
    gs = sv.make_gates([("h", (0,), ()), ("swap", (0, 5), ())])
    with sv.StateVector(8, "c64") as s:
        with pytest.raises(sv.SVError):
            sv.Batch([s], [gs], chunk_bits=6)


def test_autotune_returns_a_valid_fast_choice(sv):
    n = 20
    desc = cg.random_layers(n, 10, 2)
    gates = sv.make_gates(desc)
    best, ms = sv.autotune(n, gates, "c64")
    assert ms > 0
    assert 11 <= best["chunk_bits"] <= 13
    # the chosen options execute correctly
    with sv.StateVector(n, "c64") as st:
        st.init_basis(0)
        st.apply(gates, sv.Plan(n, gates, **best))
        st.synchronize()
        assert_close(st.get_state(), sim.simulate(n, desc), "c64")


def test_batch_tune_then_run(sv):
    """The batch tuner picks chunk bits by timing runs on the states; re-initialised states then
    give the oracle's result with the chosen options, and the byte count matches the sweeps."""
    ns, descs = _workload([12, 15, 17, 14], 16, 1e-2, 9, hea_n=16, hea_sets=2)
    gates = [sv.make_gates(d) for d in descs]
    states = [sv.StateVector(n, "c64") for n in ns]
    try:
        for s in states:
            s.init_basis(0)
        best, ms = sv.batch_tune(states, gates)
        assert ms > 0 and 10 <= best["chunk_bits"] <= 13
        b = sv.Batch(states, gates, **best)
        items, sections, nbytes = b.info()
        assert nbytes >= 16.0 * sum(2 ** n for n in ns)
        for s in states:
            s.init_basis(0)
        b.run(use_graph=True)
        b.synchronize()
        b.close()
        for n, d, s in zip(ns, descs, states):
            assert_close(s.get_state(), sim.simulate(n, d), "c64")
    finally:
        for s in states:
            s.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_from_zero_ignores_prior_contents(sv, use_graph):
    """SV_BATCH_FROM_ZERO: the first section synthesises |0..0>, so whatever the buffers held
    before does not matter; a state with an empty gate list is reset to |0..0>."""
    ns, descs = _workload([9, 14, 16, 13], 14, 2e-2, 21, hea_n=12, hea_sets=1)
    ns.append(7)
    descs.append([])
    gates = [sv.make_gates(d) for d in descs]
    rng = np.random.Generator(np.random.PCG64(5))
    states = [sv.StateVector(n, "c64") for n in ns]
    try:
        b = sv.Batch(states, gates, chunk_bits=11)
        for rep in range(2):
            for n, s in zip(ns, states):
                junk = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(np.complex64)
                s.set_state(junk)
            b.run(use_graph=use_graph, from_zero=True)
            b.synchronize()
        b.close()
        for n, d, s in zip(ns, descs, states):
            assert_close(s.get_state(), sim.simulate(n, d), "c64")
    finally:
        for s in states:
            s.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_tensor_core_sections(sv, use_graph):
    """use_tc: sections with chunks of >= 11 bits run as fused tensor-core groups (per-row norm
    restoration), smaller states stay on the SIMT groups, all in the same launch."""
    ns, descs = _workload([8, 12, 14, 16, 11, 13, 17], 12, 0.02, 31, hea_n=15, hea_sets=2)
    out, (items, sections, _) = _run_batch(sv, ns, descs, use_graph, repeats=2, chunk_bits=13, use_tc=1)
    for n, d, got in zip(ns, descs, out):
        assert_close(got, sim.simulate(n, d), "c64")


def test_batch_tensor_core_multi_section_from_zero(sv):
    ns, descs = _workload([18, 20, 15], 20, 1e-2, 41, hea_n=20, hea_sets=2)
    gates = [sv.make_gates(d) for d in descs]
    states = [sv.StateVector(n, "c64") for n in ns]
    try:
        b = sv.Batch(states, gates, chunk_bits=12, use_tc=1)
        b.run(use_graph=True, from_zero=True)
        b.synchronize()
        b.close()
        for n, d, s in zip(ns, descs, states):
            got = s.get_state()
            assert_close(got, sim.simulate(n, d), "c64")
            assert abs(float(np.vdot(got.astype(np.complex128), got.astype(np.complex128)).real) - 1.0) < 1e-6
    finally:
        for s in states:
            s.close()


@pytest.mark.parametrize("chunk_bits", [12, 13])
def test_batch_tensor_cores_requested_long_simt_programs(sv, chunk_bits):
    """Tensor cores requested, but every state fits a chunk of fewer than 11 bits, so every
    section stays on SIMT groups and the SIMT kernel runs: program pieces of long circuits
    (300+ gates in one residency) must fit its buffer."""
    ns = [9, 10, 8]
    descs = [cg.random_layers(n, 40, 50 + n) for n in ns]
    out, (items, sections, _) = _run_batch(sv, ns, descs, False, chunk_bits=chunk_bits, use_tc=1)
    assert sections == len(ns)
    for n, d, got in zip(ns, descs, out):
        assert len(d) > 300
        assert_close(got, sim.simulate(n, d), "c64")

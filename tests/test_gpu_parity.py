"""GPU parity: the CUDA library (per-gate and cache-blocked paths, through the C ABI) against the
CPU oracle, element by element.  Tolerances: complex128 1e-12 max-abs; complex64 1e-5 max-abs
and 1 - fidelity <= 1e-8."""
import math

import numpy as np
import pytest

import circuitgen as cg
from oracle import sim

from gpu_util import assert_close

pytestmark = pytest.mark.gpu

DTYPES = ["c128", "c64"]


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2102_02957_gb300 as m
    return m


def _mixed(n, count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    g = []
    for _ in range(count):
        r = int(rng.integers(0, 12))
        q = [int(v) for v in rng.permutation(n)[:2]] + [0]
        if n < 2:
            r = r % 7
        a = [float(v) for v in rng.uniform(-math.pi, math.pi, 3)]
        one = [("u3", (q[0],), tuple(a)), ("h", (q[0],), ()), ("x", (q[0],), ()), ("y", (q[0],), ()),
               ("z", (q[0],), ()), ("ry", (q[0],), (a[0],)), ("rz", (q[0],), (a[1],))]
        if r < 7:
            g.append(one[r])
        else:
            two = [("cx", (q[0], q[1]), ()), ("cz", (q[0], q[1]), ()), ("cp", (q[0], q[1]), (a[2],)),
                   ("swap", (q[0], q[1]), ()), ("unitary", (q[0], q[1]), (cg.haar_unitary(rng),))]
            g.append(two[r - 7])
    return g


def _run(sv, n, desc, dtype, basis=0, plan_opts=None):
    gates = sv.make_gates(desc)
    with sv.StateVector(n, dtype) as st:
        st.init_basis(basis)
        plan = sv.Plan(n, gates, **plan_opts) if plan_opts is not None else None
        st.apply(gates, plan)
        st.synchronize()
        return st.get_state()


@pytest.mark.parametrize("dtype", DTYPES)
def test_per_gate_random_layers_16(sv, dtype):
    desc = cg.build("rl16")
    ref = sim.simulate(16, desc)
    assert_close(_run(sv, 16, desc, dtype), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_blocked_random_layers_16(sv, dtype):
    desc = cg.build("rl16")
    ref = sim.simulate(16, desc)
    assert_close(_run(sv, 16, desc, dtype, plan_opts=dict(chunk_bits=10)), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13])
def test_per_gate_mixed(sv, dtype, n):
    desc = _mixed(n, 60, 7 * n)
    ref = sim.simulate(n, desc, 1 % (1 << n))
    assert_close(_run(sv, n, desc, dtype, basis=1 % (1 << n)), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,c", [(4, 4), (6, 4), (9, 5), (11, 8), (14, 4), (14, 13), (17, 9), (17, 13)])
@pytest.mark.parametrize("reserve", [0, 1])
def test_blocked_mixed(sv, dtype, n, c, reserve):
    desc = _mixed(n, 120, 100 + n + c) + cg.quantum_volume(n, 3, n) + cg.qft(n)
    ref = sim.simulate(n, desc, 3)
    assert_close(_run(sv, n, desc, dtype, basis=3, plan_opts=dict(chunk_bits=c, reserve=reserve)), ref, dtype)


@pytest.mark.parametrize("dtype,n,c,pinned", [("c128", 22, 13, 0), ("c64", 22, 14, 0), ("c128", 22, 13, 4),
                                              ("c64", 23, 13, 0)])
def test_blocked_wide_chunks_many_per_block(sv, dtype, n, c, pinned):
    """Chunks so wide that fewer shared-memory buffers than consumer groups fit (128 KiB chunks:
    one buffer) or only one spare (64 KiB), with hundreds of chunks, so every thread block works
    through several of them: the buffer hand-over between consumer groups is exercised."""
    desc = cg.random_layers(n, 6, 900 + c) + cg.quantum_volume(n, 2, 901)
    ref = sim.simulate(n, desc, 5)
    got = _run(sv, n, desc, dtype, basis=5, plan_opts=dict(chunk_bits=c, gather_pinned=pinned))
    assert_close(got, ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,c", [(12, 6), (16, 10)])
def test_blocked_keep_layout(sv, dtype, n, c):
    desc = cg.random_layers(n, 4, 5) + [("swap", (0, n - 1), ())] + cg.quantum_volume(n, 2, 6)
    gates = sv.make_gates(desc)
    plan = sv.Plan(n, gates, chunk_bits=c, restore_layout=False)
    fmap = list(plan.info().final_map[:n])
    with sv.StateVector(n, dtype) as st:
        st.init_basis(0)
        st.apply(gates, plan)
        got = st.get_state()
    idx = np.arange(1 << n)
    phys = np.zeros_like(idx)
    for q in range(n):
        phys |= ((idx >> q) & 1) << fmap[q]
    assert_close(got[phys], sim.simulate(n, desc), dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [11, 14, 20])
def test_output_reordering_only(sv, dtype, n):
    # SWAP relabels only: the blocked path must realise the bit permutation with the
    # reordering rounds (low-low, low-high and high-high pairs)
    rng = np.random.Generator(np.random.PCG64(n))
    desc = [("h", (q,), ()) for q in range(0, n, 3)] + [("ry", (q,), (0.1 * q,)) for q in range(n)]
    for _ in range(3 * n):
        a, b = (int(v) for v in rng.permutation(n)[:2])
        desc.append(("swap", (a, b), ()))
    desc.append(("u3", (1,), (0.3, 0.2, 0.1)))
    ref = sim.simulate(n, desc, 5)
    assert_close(_run(sv, n, desc, dtype, basis=5, plan_opts=dict(chunk_bits=6)), ref, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [16, 22])
def test_qft_closed_form(sv, dtype, n):
    x = cg.basis_index(n, 2)
    y = np.arange(1 << n)
    ref = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    desc = cg.qft(n)
    assert_close(_run(sv, n, desc, dtype, basis=x), ref, dtype)
    assert_close(_run(sv, n, desc, dtype, basis=x, plan_opts=dict(chunk_bits=10)), ref, dtype)


# ------------------------------------------------------------------ readouts

@pytest.mark.parametrize("dtype", DTYPES)
def test_probabilities_norm_expval(sv, dtype):
    import torch
    n = 12
    desc = cg.random_layers(n, 6, 11)
    ref = sim.simulate(n, desc)
    gates = sv.make_gates(desc)
    tol = 1e-12 if dtype == "c128" else 1e-5
    with sv.StateVector(n, dtype) as st:
        st.init_basis(0)
        st.apply(gates, sv.Plan(n, gates, chunk_bits=8))
        p = st.probabilities()
        assert np.abs(p - sim.probabilities(ref)).max() < tol
        pd = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        st.probabilities(pd)
        assert np.abs(pd.cpu().numpy() - p).max() == 0
        assert abs(st.norm2() - 1) < (1e-12 if dtype == "c128" else 1e-5)
        for x, z in cg.random_pauli_strings(n, 12, 4) + [(0, 0), (0, 1), (4095, 0)]:
            e = st.expval_pauli(x, z)
            r = sim.expval_pauli(ref, x, z)
            assert abs(e - r) < tol, (x, z, e, r)


@pytest.mark.parametrize("dtype", DTYPES)
def test_sample_exact_dyadic(sv, dtype):
    n = 20
    ghz = [("h", (0,), ())] + [("cx", (q, q + 1), ()) for q in range(n - 1)]
    gates = sv.make_gates(ghz)
    with sv.StateVector(n, dtype) as st:
        st.init_basis(0)
        st.apply(gates, sv.Plan(n, gates, chunk_bits=8))
        s = st.sample(5000, 99)
    ref = sim.sample(sim.probabilities(sim.simulate(n, ghz)), 5000, 99)
    assert np.array_equal(s, ref)
    with sv.StateVector(n, dtype) as st:
        st.init_basis(123457)
        assert np.all(st.sample(1000, 3) == 123457)


def test_sample_distribution(sv):
    n = 8
    desc = cg.random_layers(n, 4, 6)
    gates = sv.make_gates(desc)
    with sv.StateVector(n, "c128") as st:
        st.init_basis(0)
        st.apply(gates)
        s = st.sample(100000, 5)
    p = sim.probabilities(sim.simulate(n, desc))
    # same uniforms and an exact-enough cumsum: almost every shot agrees with the oracle
    ref = sim.sample(p, 100000, 5)
    assert np.mean(s == ref) > 0.999
    counts = np.bincount(s.astype(np.int64), minlength=1 << n)
    exp = p * 100000
    keep = exp > 5
    assert (((counts - exp) ** 2)[keep] / exp[keep]).sum() < 400


# ------------------------------------------------------------------ errors

def test_plan_mismatch_rejected(sv):
    n = 10
    a = sv.make_gates(cg.random_layers(n, 2, 1))
    b = sv.make_gates(cg.random_layers(n, 2, 2))
    plan = sv.Plan(n, a, chunk_bits=6)
    with sv.StateVector(n, "c64") as st:
        st.init_basis(0)
        with pytest.raises(sv.SVError) as e:
            st.apply(b, plan)
        assert e.value.status == sv._lib.SV_ERR_PLAN
    with sv.StateVector(n + 1, "c64") as st:
        with pytest.raises(sv.SVError) as e:
            st.apply(a, plan)
        assert e.value.status in (sv._lib.SV_ERR_PLAN, sv._lib.SV_ERR_ARG)


def test_bad_arguments(sv):
    with pytest.raises(sv.SVError):
        sv.StateVector(40, "c64")
    with sv.StateVector(5, "c64") as st:
        with pytest.raises(sv.SVError):
            st.init_basis(1 << 5)
        with pytest.raises(sv.SVError):
            st.expval_pauli(1 << 6, 0)


def test_torch_buffer_and_stream(sv):
    import torch
    n = 14
    buf = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    desc = cg.quantum_volume(n, 5, 3)
    gates = sv.make_gates(desc)
    with sv.StateVector(n, "c64", buffer=buf, stream=s) as st:
        st.init_basis(0)
        st.apply(gates, sv.Plan(n, gates, chunk_bits=9))
        st.synchronize()
        assert st.device_ptr() == buf.data_ptr()
    got = torch.view_as_complex(buf.view(-1, 2)).cpu().numpy()
    assert_close(got, sim.simulate(n, desc), "c64")


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,c,pinned", [(10, 6, 4), (12, 8, 4), (17, 10, 4), (20, 13, 4), (18, 12, 5), (14, 12, 4)])
def test_gathered_chunks_mixed(sv, dtype, n, c, pinned):
    desc = _mixed(n, 100, 300 + n + c) + cg.quantum_volume(n, 4, n + 1) + cg.qft(n)
    ref = sim.simulate(n, desc, 11)
    got = _run(sv, n, desc, dtype, basis=11, plan_opts=dict(chunk_bits=c, gather_pinned=pinned))
    assert_close(got, ref, dtype)


@pytest.mark.parametrize("seg_bits", [4, 5])
def test_gathered_quantum_volume_24(sv, seg_bits):
    n = 24
    desc = cg.quantum_volume(n, 8, 17)
    ref = sim.simulate(n, desc)
    got = _run(sv, n, desc, "c64", plan_opts=dict(chunk_bits=13, gather_pinned=4, seg_bits=seg_bits))
    assert_close(got, ref, "c64")


def test_chunk_larger_than_shared_memory_rejected(sv):
    n = 16
    gates = sv.make_gates(cg.quantum_volume(n, 2, 1))
    for opts in (dict(chunk_bits=16), dict(chunk_bits=16, gather_pinned=4)):
        with sv.StateVector(n, "c64") as st:
            st.init_basis(0)
            with pytest.raises(sv.SVError) as e:
                st.apply(gates, sv.Plan(n, gates, **opts))
            assert e.value.status == sv._lib.SV_ERR_UNSUPPORTED


# ------------------------------------------------------------------ tensor-core fused groups (3xTF32)

@pytest.mark.parametrize("n,c,pinned", [(14, 11, 0), (16, 12, 0), (17, 13, 0), (16, 11, 4), (20, 12, 4), (20, 13, 4), (13, 13, 0), (12, 12, 0)])
def test_tensor_core_fused_groups(sv, n, c, pinned):
    desc = _mixed(n, 150, 500 + n + c) + cg.quantum_volume(n, 6, n + 2) + cg.qft(n)
    ref = sim.simulate(n, desc, 9)
    got = _run(sv, n, desc, "c64", basis=9, plan_opts=dict(chunk_bits=c, gather_pinned=pinned, use_tc=1))
    assert_close(got, ref, "c64")


def test_tensor_core_many_groups_per_section(sv):
    # a single section with far more register groups than fit beside the chunk ring: split
    # into several sweeps over the same chunks
    n = 13
    desc = cg.quantum_volume(n, 40, 3)
    ref = sim.simulate(n, desc)
    got = _run(sv, n, desc, "c64", plan_opts=dict(chunk_bits=13, use_tc=1))
    assert_close(got, ref, "c64")


@pytest.mark.parametrize("c", [12, 13])
def test_tensor_core_quantum_volume_24(sv, c):
    # 12-bit chunks run four single-buffered consumer groups, 13-bit ones two double-buffered
    n = 24
    desc = cg.quantum_volume(n, 10, 19)
    ref = sim.simulate(n, desc)
    got = _run(sv, n, desc, "c64", plan_opts=dict(chunk_bits=c, gather_pinned=4, use_tc=1))
    assert_close(got, ref, "c64")


@pytest.mark.parametrize("r", [3, 4, 5])
@pytest.mark.parametrize("n,c,pinned", [(12, 12, 0), (14, 12, 0), (20, 12, 4), (24, 12, 5), (17, 13, 0), (21, 13, 4)])
def test_tensor_core_group_widths(sv, r, n, c, pinned):
    """Fused groups of r = 3, 4 and 5 bits (8x8, 16x16 and 32x32 unitaries; real embeddings of
    K = 16, 32, 64) applied as 3xTF32 MMAs, with and without the per-circuit norm restoration,
    against the oracle: single-chunk, contiguous (chunk_swap) and gathered layouts."""
    desc = _mixed(n, 120, 700 + n + c + r) + cg.quantum_volume(n, 6, n + r)
    ref = sim.simulate(n, desc, 5)
    for raw in (0, 1):
        got = _run(sv, n, desc, "c64", basis=5,
                   plan_opts=dict(chunk_bits=c, gather_pinned=pinned, use_tc=1, seg_bits=r, tc_no_renorm=raw))
        assert_close(got, ref, "c64")


def test_tensor_core_width_needs_room(sv):
    """A 5-bit tensor-core group needs 128 rows of 32 amplitudes: with 11-bit chunks the plan runs on
    SIMT register groups of 5 bits instead, still on the GPU and still exact to the tolerance."""
    n = 14
    desc = cg.quantum_volume(n, 2, 1)
    gates = sv.make_gates(desc)
    with sv.StateVector(n, "c64") as st:
        st.init_basis(0)
        plan = sv.Plan(n, gates, chunk_bits=11, use_tc=1, seg_bits=5)
        st.apply(gates, plan)
        st.synchronize()
        assert_close(st.get_state(), sim.simulate(n, desc), "c64")


def _diag_rich(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for g in cg.random_layers(n, 3, seed):
        out.append(g)
        a, b = (int(v) for v in rng.permutation(n)[:2])
        out.append([("cz", (a, b), ()), ("cp", (a, b), (float(rng.uniform(0, 6.3)),)),
                    ("rz", (a,), (float(rng.uniform(0, 6.3)),)), ("z", (b,), ())][int(rng.integers(0, 4))])
    return out


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,c,pinned", [(12, 6, 0), (16, 10, 0), (16, 10, 4), (13, 8, 3), (20, 12, 4), (14, 5, 1)])
def test_diag_outside_sections(sv, dtype, n, c, pinned):
    """Diagonal gates applied inside sections whose chunk lacks some of their qubits (the chunk's
    fixed bits select the diagonal): QFT of a basis state, a CZ-ladder ansatz and random layers
    with CZ/CP/RZ/Z, both chunk layouts, against the oracle."""
    x = cg.basis_index(n, 2)
    for desc in (cg.qft(n), cg.hea(n, 3, n, 1), _diag_rich(n, n + c)):
        ref = sim.simulate(n, desc, x)
        assert_close(_run(sv, n, desc, dtype, basis=x,
                          plan_opts=dict(chunk_bits=c, gather_pinned=pinned, diag_outside=1)), ref, dtype)


def test_async_state_copies_on_two_streams(sv):
    """sv_set_state_async / sv_get_state_async from and to pinned host memory, two states on two
    streams taking turns (the benchmark's end-to-end pipeline), against the oracle."""
    import torch
    n, c = 20, 10
    desc = cg.quantum_volume(n, 4, 31)
    gates = sv.make_gates(desc)
    plan = sv.Plan(n, gates, chunk_bits=c)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    states = [sv.StateVector(n, "c64", stream=s) for s in streams]
    h_in = torch.zeros(1 << n, dtype=torch.complex64).pin_memory()
    h_in[5] = 1.0
    h_out = [torch.zeros(1 << n, dtype=torch.complex64).pin_memory() for _ in range(2)]
    try:
        for i in range(4):
            k = i & 1
            states[k].set_state_async(h_in.data_ptr())
            states[k].apply(gates, plan)
            states[k].get_state_async(h_out[k].data_ptr())
        for s in states:
            s.synchronize()
        ref = sim.simulate(n, desc, 5)
        for k in range(2):
            assert_close(h_out[k].numpy(), ref, "c64")
    finally:
        for s in states:
            s.close()

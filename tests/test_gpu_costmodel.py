"""The learned cost model on the GPU: forward, gradient and Adam kernels against the float64
reference (oracle/mlp.py), training, the timing collector, and the steered planner (amplitude
parity with the oracle, and its measured time against the paper's rule)."""
import numpy as np
import pytest

import circuitgen as cg
from oracle import mlp, sim

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


def _data(seed, rows):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = rng.normal(0.0, 0.3, mlp.N_PARAMS).astype(np.float32)
    X = rng.uniform(0.0, 1.0, (rows, mlp.N_IN)).astype(np.float32)
    T = rng.normal(0.0, 1.0, rows).astype(np.float32)
    return theta, X, T


@pytest.mark.parametrize("rows", [1, 7, 300])
def test_forward_matches_reference(sv, rows):
    theta, X, _ = _data(1, rows)
    cm = sv.CostModel(0)
    cm.set_params(theta)
    np.testing.assert_array_equal(cm.params(), theta)
    y = cm.forward(X)
    ref, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y - ref) / (1.0 + np.abs(ref))) < 2e-5


@pytest.mark.parametrize("rows", [1, 33, 1000])
def test_gradient_matches_reference(sv, rows):
    theta, X, T = _data(2, rows)
    cm = sv.CostModel(0)
    cm.set_params(theta)
    g, loss = cm.gradient(X, T)
    gref, lref = mlp.gradient(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert loss == pytest.approx(lref, rel=1e-5)
    assert np.max(np.abs(g - gref)) <= 1e-4 * np.max(np.abs(gref))


def test_adam_steps_match_reference(sv):
    theta, X, T = _data(3, 64)
    lr = 1e-2
    cm = sv.CostModel(0)
    cm.set_params(theta)
    th = theta.astype(np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    for step in (1, 2):
        g, _ = mlp.gradient(th, X.astype(np.float64), T.astype(np.float64))
        cm.adam_step(X, T, lr)
        th_next, m, v = mlp.adam_step(th, m, v, g, step, lr)
        got = cm.params().astype(np.float64)
        # where the gradient is not tiny the update direction is fixed: compare closely; elsewhere
        # the step is bounded by lr (Adam's per-coordinate step bound)
        big = np.abs(g) > 1e-3 * np.max(np.abs(g))
        assert np.max(np.abs(got[big] - th_next[big])) <= 2e-3 * lr
        assert np.max(np.abs(got - th)) <= 1.5 * lr
        th = got


def test_training_reduces_error(sv):
    rng = np.random.Generator(np.random.PCG64(4))
    X = rng.uniform(0.0, 1.0, (2000, 16)).astype(np.float32)
    us = np.exp(1.0 + 2.0 * X[:, 0] + np.sin(3.0 * X[:, 3]) - X[:, 5] * X[:, 6]).astype(np.float32)
    cm = sv.CostModel(5)
    cm.add_samples(X, us)
    assert cm.num_samples() == 2000
    base = float(np.var(np.log(us)))
    mse = cm.train(epochs=150, batch=128, lr=2e-3, seed=9)
    assert mse < 0.05 * base
    pred = cm.predict_us(X[:50])
    assert np.max(np.abs(np.log(pred) - np.log(us[:50]))) < 0.5


@pytest.fixture(scope="module")
def trained(sv):
    """A model trained on section timings collected at n = 24 (random-layer and quantum-volume
    circuits, several chunk sizes, SIMT and tensor-core sections, random candidate choices)."""
    n = 24
    cm = sv.CostModel(11)
    opts = [dict(chunk_bits=c, gather_pinned=4, use_tc=tc) for c in (11, 12, 13) for tc in (0, 1)]
    with sv.StateVector(n, "c64") as st:
        for k, desc in enumerate([cg.random_layers(n, 10, 40 + s) for s in range(3)] +
                                 [cg.quantum_volume(n, 8, 50 + s) for s in range(3)]):
            g = sv.make_gates(desc)
            cm.collect(st, g, opts, policy_seed=0)
            cm.collect(st, g, opts, policy_seed=1000 + 17 * k)
    assert cm.num_samples() > 300
    cm.train(epochs=300, batch=128, lr=2e-3, seed=3)
    return cm


def test_collect_adds_one_sample_per_section(sv):
    n = 18
    desc = cg.random_layers(n, 6, 8)
    g = sv.make_gates(desc)
    cm = sv.CostModel(0)
    with sv.StateVector(n, "c64") as st:
        added = cm.collect(st, g, [dict(chunk_bits=12, gather_pinned=4)])
    plan = sv.Plan(n, g, chunk_bits=12, gather_pinned=4)
    assert added == plan.info().n_blocks == cm.num_samples()


@pytest.mark.parametrize("use_tc", [0, 1])
def test_steered_plan_gives_oracle_state(sv, trained, use_tc):
    n = 20
    for desc in (cg.random_layers(n, 10, 77), cg.quantum_volume(n, 6, 78)):
        g = sv.make_gates(desc)
        plan = sv.Plan(n, g, model=trained, chunk_bits=13, gather_pinned=4, use_tc=use_tc)
        with sv.StateVector(n, "c64") as st:
            st.init_basis(0)
            st.apply(g, plan)
            st.synchronize()
            assert_close(st.get_state(), sim.simulate(n, desc), "c64")


def _sections(stream):
    """(chunk mask, gate indices) of every gathered section in a serialised library plan."""
    it = iter(stream)
    _n, _c, _reserve, _restore, nops = (next(it) for _ in range(5))
    out = []
    for _ in range(nops):
        kind = next(it)
        if kind in (1, 3):
            cnt = next(it)
            for _ in range(2 * cnt):
                next(it)
        else:
            mask = next(it) if kind == 4 else None
            cnt = next(it)
            gis = []
            for _ in range(cnt):
                gi, _nq, _p0, _p1 = next(it), next(it), next(it), next(it)
                gis.append(gi)
            out.append((mask, gis))
    return out


@pytest.mark.parametrize("use_tc", [0, 1])
def test_steered_schedule_is_one_of_the_oracle_candidates(sv, trained, use_tc):
    """Each section of a steered plan is one of the candidate chunks the oracle restates (the
    rule at the full chunk and one and two qubits smaller, and the look-ahead chunk), and given
    those choices the whole schedule equals the oracle's bit for bit.  The choice among the
    candidates is the network's and is not restated."""
    from oracle import planner
    n, c, pinned = 20, 13, 4
    for desc in (cg.random_layers(n, 10, 77), cg.quantum_volume(n, 6, 78), cg.quantum_volume(n, 10, 79)):
        g = sv.make_gates(desc)
        plan = sv.Plan(n, g, model=trained, chunk_bits=c, gather_pinned=pinned, use_tc=use_tc)
        stream = plan.serialize()
        want = [mask for mask, _ in _sections(stream)]
        picks = []

        def steer(cands):
            k = len(picks)
            masks = [sum(1 << q for q in cs) for cs in cands]
            assert k < len(want) and want[k] in masks, (k, want[k:k + 1], masks)
            picks.append(masks.index(want[k]))
            return picks[-1]

        q = planner.plan_blocking(n, desc, c, pinned=pinned, steer=steer,
                                  steer_min_chunk=max(pinned + 2, 4 + 7 if use_tc else 1))
        assert q.serialize() == stream
        print(f"use_tc={use_tc}: {len(picks)} sections, candidate picked per section {picks}")


def _time_ms(sv, st, g, plan, reps=5):
    import torch
    ts = []
    for _ in range(reps):
        st.init_basis(0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st.apply(g, plan)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def test_steered_planner_gain_on_held_out_circuits(sv, trained):
    """Held-out circuits at n = 26: the steered plan's measured time (median of 5 runs) against the
    paper's rule and against the look-ahead chunk choice, same options.  The steered planner must
    beat the rule by more than timing noise (2 %); its standing against look-ahead is printed."""
    n = 26
    rows = []
    with sv.StateVector(n, "c64") as st:
        for desc in (cg.random_layers(n, 12, 901), cg.quantum_volume(n, 10, 902)):
            g = sv.make_gates(desc)
            for tc in (0, 1):
                o = dict(chunk_bits=13, gather_pinned=4, use_tc=tc)
                rule = sv.Plan(n, g, **o)
                look = sv.Plan(n, g, lookahead=1, **o)
                steer = sv.Plan(n, g, model=trained, **o)
                t_rule = _time_ms(sv, st, g, rule)
                t_look = _time_ms(sv, st, g, look)
                t_steer = _time_ms(sv, st, g, steer)
                rows.append((tc, rule.info().n_blocks, look.info().n_blocks, steer.info().n_blocks, t_rule, t_look,
                             t_steer))
    for tc, nb_r, nb_l, nb_s, tr, tl, ts in rows:
        print(f"tc={tc} sections rule={nb_r} look-ahead={nb_l} steered={nb_s}  ms rule={tr:.3f} "
              f"look-ahead={tl:.3f} steered={ts:.3f}  gain vs rule {tr / ts:.3f}x, vs look-ahead {tl / ts:.3f}x")
    total_rule = sum(r[4] for r in rows)
    total_look = sum(r[5] for r in rows)
    total_steer = sum(r[6] for r in rows)
    print(f"total gain vs rule {total_rule / total_steer:.3f}x, vs look-ahead {total_look / total_steer:.3f}x")
    assert total_steer <= 0.98 * total_rule


def test_steered_section_widths_give_oracle_state(sv):
    """A steered plan picks each section's register-group width (4 or 5 bits) by the network's
    predicted time; networks fitted briefly to random timings (several seeds) choose differently
    from section to section, and a plan mixing both widths must still give the oracle's state."""
    n = 20
    desc = cg.quantum_volume(n, 10, 81)
    g = sv.make_gates(desc)
    mixed = None
    for seed in range(12):
        rng = np.random.Generator(np.random.PCG64(100 + seed))
        cm = sv.CostModel(seed)
        cm.add_samples(rng.uniform(0.0, 1.0, (64, 16)).astype(np.float32),
                       np.exp(rng.normal(5.0, 1.0, 64)).astype(np.float32))
        cm.train(epochs=2, batch=32, lr=1e-3, seed=seed)
        plan = sv.Plan(n, g, model=cm, chunk_bits=13, gather_pinned=4, use_tc=1)
        w = set(int(x) for x in plan.widths())
        assert w <= {4, 5}
        if w == {4, 5}:
            mixed = plan
            break
    assert mixed is not None, "no seed gave a plan with both widths"
    with sv.StateVector(n, "c64") as st:
        st.init_basis(0)
        st.apply(g, mixed)
        st.synchronize()
        assert_close(st.get_state(), sim.simulate(n, desc), "c64")
    assert mixed.info().n_segments > 0

"""The failure path of the bounded device waits, without faulting or hanging the GPU: a batch
whose first state's first section never releases the later ones (SV_BATCH_TEST_STALL, a flag
nothing in normal operation sets) with a short wait bound.  The launch gives up after the bound,
the host sees SV_ERR_TIMEOUT, and the context stays usable: the same batch then runs correctly."""
import time

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


@pytest.mark.parametrize("use_tc", [0, 1])
def test_stalled_batch_times_out_and_the_device_recovers(sv, use_tc):
    ns = [16, 14, 15]
    descs = [cg.noisy_trajectory(n, 12, 0.01, 21, t) for t, n in enumerate(ns)]
    gates = [sv.make_gates(d) for d in descs]
    states = [sv.StateVector(n, "c64") for n in ns]
    b = sv.Batch(states, gates, chunk_bits=11, use_tc=use_tc, wait_limit_ms=200)
    try:
        assert b.info()[1] > len(ns)  # several sections per state: there is a later section to stall
        t0 = time.time()
        b.run(from_zero=True, test_stall=True)
        with pytest.raises(sv.SVError) as e:
            b.synchronize()
        waited = time.time() - t0
        assert e.value.status == sv._lib.SV_ERR_TIMEOUT
        assert waited < 30.0, waited
        # the error word is cleared by the report; the next run is complete and correct
        b.run(from_zero=True)
        b.synchronize()
        for n, d, s in zip(ns, descs, states):
            assert_close(s.get_state(), sim.simulate(n, d), "c64")
    finally:
        b.close()
        for s in states:
            s.close()


def test_stall_flag_refused_with_graph(sv):
    n = 14
    desc = cg.random_layers(n, 4, 3)
    st = sv.StateVector(n, "c64")
    b = sv.Batch([st], [sv.make_gates(desc)], chunk_bits=10)
    try:
        with pytest.raises(sv.SVError) as e:
            b.run(use_graph=True, test_stall=True)
        assert e.value.status == sv._lib.SV_ERR_ARG
    finally:
        b.close()
        st.close()

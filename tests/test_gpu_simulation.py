"""Parity of the device discrete-event simulation with queueing (one launch
for the whole run) with the oracle: start steps, every request's result
(attempts' decisions included) and the final state bit-exact, for the four
methods, one block and a cluster.  Needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W
from parity_util import assert_same_result, assert_same_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched

    dcsched.lib()
    return dcsched


@pytest.fixture(scope="module")
def stream():
    import torch

    return torch.cuda.Stream()


def _check(ds, stream, wl, sub, dur, T, where):
    inst = wl.instances[0]
    reqs = [inst.reqs.request(r) for r in range(inst.reqs.n)]
    dc = ds.load_instance(inst, stream=stream)
    start = dc.simulate(T, sub, dur)
    odc = O.OracleDC.from_instance(inst)
    outs, ostart = odc.simulate(reqs, sub, dur, T)
    assert np.array_equal(start, ostart), where
    for r in range(inst.reqs.n):
        assert_same_result(dc.query(r), outs[r], "%s req %d" % (where, r))
    assert_same_state(dc, odc, where)
    return start


@pytest.mark.parametrize("method", [W.TOPSIS, W.AHP, W.BF, W.WF])
def test_simulation_heavy_queue(ds, stream, method):
    T = 150
    wl, sub, dur = W.simulation(seed=21, k=4, n_requests=200, n_steps=T, max_duration=40,
                                host_cpu=8, host_mem=16, link_mbps=100, method=method)
    start = _check(ds, stream, wl, sub, dur, T, "sim heavy m%d" % method)
    assert np.sum(start < 0) > 0 and np.sum(start > sub) > 0  # it queued


def test_simulation_k8_cluster(ds, stream):
    T = 200
    wl, sub, dur = W.simulation(seed=22, k=8, n_requests=500, n_steps=T, max_duration=80,
                                host_cpu=8, host_mem=16, link_mbps=200)
    inst = wl.instances[0]
    key = (inst.k, inst.n_criteria, inst.method, inst.pair_rule)
    ds.set_launch(*key, 256, 2)
    try:
        _check(ds, stream, wl, sub, dur, T, "sim k8 cluster")
    finally:
        ds.set_launch(*key, 0, 1)


def test_simulation_rejects_queued_departures(ds, stream):
    inst = W.small().instances[0]
    dc = ds.DataCenter.from_instance(inst, stream=stream)
    dc.submit(inst.reqs.request(0))
    ds.schedule([dc])
    dc.submit(inst.reqs.request(1))
    dc.release(0)
    with pytest.raises(ds.DcError):
        dc.simulate(10, [0], [1])

"""Serving with continuous batching (dc_server): timed Poisson arrivals over
several resident data centers, departures in each data center's FCFS
stream, admission under a device-memory budget.  Every result equals the
FP64 oracle's FCFS run of its data center and the result of that data center
scheduled alone; the one-request-per-launch mode gives the same results.
Needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W
from parity_util import assert_same_result

pytestmark = pytest.mark.gpu


def _served(ds, wl, max_per_launch, admit_bytes):
    import torch

    dcs = [ds.DataCenter.from_instance(inst, stream=torch.cuda.Stream()) for inst in wl.instances]
    t, inst, kind, local, rel = W.serving_events(wl)
    reqs = [wl.instances[inst[e]].reqs.request(int(local[e])) if kind[e] == 0 else None
            for e in range(len(t))]
    srv = ds.Server(dcs, admit_bytes=admit_bytes, max_requests_per_launch=max_per_launch)
    lat, rid, stats = srv.replay(t, inst, kind, reqs, rel)
    return dcs, (t, inst, kind, local, rel), lat, rid, stats


@pytest.mark.parametrize("max_per_launch,admit_bytes", [(0, 1 << 30), (0, 40000), (1, 1 << 30)])
def test_served_results_equal_oracle_and_alone(max_per_launch, admit_bytes):
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched as ds

    wl = W.serving(n_instances=5, rate_per_s=20000.0, duration_s=0.012, k=8, size_hi=24,
                   mean_life=6.0)
    dcs, (t, inst, kind, local, rel), lat, rid, stats = _served(ds, wl, max_per_launch, admit_bytes)
    n_req = int((kind == 0).sum())
    assert stats["requests"] == n_req and n_req > 100
    assert np.all(lat[kind == 0] >= 0)
    if max_per_launch == 1:
        # one request per launch (launches holding only departures add to it)
        assert stats["launches"] >= n_req
    else:
        assert stats["launches"] < n_req  # requests were batched
    if admit_bytes < (1 << 20):
        assert stats["peak_admitted_bytes"] <= max(admit_bytes, 40000)
    for i, ins in enumerate(wl.instances):
        ref, _ = O.run_instance(ins)
        alone = ds.load_instance(ins)
        ds.schedule([alone])
        for e in np.nonzero((kind == 0) & (inst == i))[0]:
            j = int(local[e])
            got = dcs[i].query(int(rid[e]))
            assert_same_result(got, ref[j], "served inst %d req %d" % (i, j))
            assert_same_result(got, alone.query(j), "served vs alone inst %d req %d" % (i, j))
        alone.close()
    for d in dcs:
        d.close()


def test_replay_stall_returns_timeout():
    """The replay's bounded wait: one request of 60,000 zero-size singleton
    pods on a k=16 data center is a single operation of ~0.7 s on the device
    (a pod decision is ~11 us), during which the kernel reports no progress;
    with a 0.1 s stall limit the replay returns DC_E_TIMEOUT once the launch
    has finished, and the library keeps working afterwards."""
    import torch
    from paper_1909_07673_gb300 import dcsched as ds

    torch.cuda.set_device(0)
    n = 60000
    z = np.zeros(n, np.int32)
    e = np.zeros(0, np.int32)
    big = {"cpu_min": z, "cpu_max": z, "mem_min": z, "mem_max": z,
           "pod": np.arange(n, dtype=np.int32), "src": e, "dst": e, "bw_min": e, "bw_max": e}
    dc = ds.DataCenter(16, 32, 64, 10000, 6, ds.TOPSIS, ds.RATIO, (1 / 6,) * 6,
                       stream=torch.cuda.Stream())
    srv = ds.Server([dc], stall_s=0.1)
    with pytest.raises(ds.DcError) as ei:
        srv.replay(np.zeros(1), np.zeros(1, np.int32), np.zeros(1, np.int32), [big],
                   np.zeros(1, np.int32))
    assert ei.value.code == ds.E_TIMEOUT
    srv.close()
    dc.close()
    with pytest.raises(ds.DcError):
        ds.Server([], stall_s=1.0)
    # a fresh data center schedules normally after the timeout
    inst = W.small().instances[0]
    fresh = ds.load_instance(inst, stream=torch.cuda.Stream())
    ds.schedule([fresh])
    ref, _ = O.run_instance(inst)
    for r in range(inst.reqs.n):
        assert_same_result(fresh.query(r), ref[r], "after timeout req %d" % r)
    fresh.close()

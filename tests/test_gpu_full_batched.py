"""The full batched workload (256 fat-tree data centers, k 8/16/24/32, 100
requests of 4-256 containers each, TOPSIS, 6 criteria) in the launch
configuration the benchmark times: one captured plan with a state reset,
launched twice.  For one data center of every size the first requests are
compared element by element with the oracle; for every eighth data center
the invariants that hold at any size are checked (final free CPU, memory and
link residuals equal capacity minus pre-load minus what the accepted
requests hold; allocations inside their intervals; rejected requests hold
nothing); every data center's state stays non-negative.  Needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W
from parity_util import assert_same_result

pytestmark = pytest.mark.gpu

PREFIX = 5


@pytest.fixture(scope="module")
def ds():
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched

    dcsched.lib()
    return dcsched


def _invariants(ds, dc, inst):
    H = inst.hosts
    used_c = np.zeros(H, np.int64)
    used_m = np.zeros(H, np.int64)
    used_l = np.zeros(3 * H, np.int64)
    for r in range(inst.reqs.n):
        out = dc.query(r)
        q = inst.reqs.request(r)
        if out["status"] == ds.ACCEPTED:
            assert np.all(out["host"] >= 0) and np.all(out["host"] < H)
            np.add.at(used_c, out["host"], out["cpu"])
            np.add.at(used_m, out["host"], out["mem"])
            assert np.all((out["cpu"] >= q["cpu_min"]) & (out["cpu"] <= q["cpu_max"]))
            assert np.all((out["mem"] >= q["mem_min"]) & (out["mem"] <= q["mem_max"]))
            for e in range(len(q["src"])):
                links = out["path"][6 * e:6 * e + 6]
                np.add.at(used_l, links[links >= 0], out["bw"][e])
        else:
            assert out["status"] == ds.REJECTED
            assert np.all(out["host"] == -1) and np.all(out["cpu"] == 0)
    assert np.array_equal(dc.state(ds.FREE_CPU), inst.host_cpu - inst.pre_cpu - used_c)
    assert np.array_equal(dc.state(ds.FREE_MEM), inst.host_mem - inst.pre_mem - used_m)
    assert np.array_equal(dc.state(ds.LINK_RES), inst.link_mbps - inst.pre_link - used_l)


def test_full_batched_sampled(ds):
    import torch

    stream = torch.cuda.Stream()
    wl = W.batched()
    dcs = [ds.load_instance(inst, stream=stream) for inst in wl.instances]
    plan = ds.Plan(dcs, ds.PLAN_GRAPH | ds.PLAN_RESET)
    for _ in range(2):  # the replay after a reset gives the same results
        plan.launch(stream)
        torch.cuda.synchronize()
    plan.collect()
    dec, hr, _, _ = plan.stats()
    assert dec > 0 and hr > 0
    seen = set()
    for i, (dc, inst) in enumerate(zip(dcs, wl.instances)):
        if inst.k in seen:
            continue
        seen.add(inst.k)
        ref, _ = O.run_instance(inst, max_requests=PREFIX)
        for r in range(PREFIX):
            assert_same_result(dc.query(r), ref[r], "batched inst %d (k=%d) req %d" % (i, inst.k, r))
    for i in range(0, len(dcs), 8):
        _invariants(ds, dcs[i], wl.instances[i])
    for dc in dcs:
        for f in (ds.FREE_CPU, ds.FREE_MEM, ds.LINK_RES):
            assert np.all(dc.state(f) >= 0)
    plan.close()
    for dc in dcs:
        dc.close()

"""The full batched workload (256 fat-tree data centers, k 8/16/24/32, 100
requests of 4-256 containers each, TOPSIS, 6 criteria) in the launch
configuration the benchmark times: launch shapes chosen by the autotuner
on all operations of every data center, one captured plan with a state
reset, launched twice.  Every request of every data center (25,600 requests,
about 1.6 million pod decisions) and every data center's final state are
compared element by element with the oracle, which runs over a pool of host
threads (one data center per task); every eighth data center is also
checked against the invariants that hold at any size (final free CPU,
memory and link residuals equal capacity minus pre-load minus what the
accepted requests hold; allocations inside their intervals; rejected
requests hold nothing).  Needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W
from parity_util import compare_chains, gpu_results

pytestmark = pytest.mark.gpu



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


def test_full_batched_whole_chains(ds):
    import torch

    stream = torch.cuda.Stream()
    wl = W.batched()
    dcs = [ds.load_instance(inst, stream=stream) for inst in wl.instances]
    tuned = ds.autotune(dcs, max_ops=0)
    try:
        plan = ds.Plan(dcs, ds.PLAN_GRAPH | ds.PLAN_RESET)
        for _ in range(2):  # the replay after a reset gives the same results
            plan.launch(stream)
            torch.cuda.synchronize()
        plan.collect()
    finally:
        for e in tuned:  # back to the default shapes for the other tests
            ds.set_launch(e["k"], e["n_criteria"], e["method"], e["pair_rule"], 0, 1)
    dec, hr, _, _ = plan.stats()
    assert dec > 0 and hr > 0
    jobs = []
    for i, (dc, inst) in enumerate(zip(dcs, wl.instances)):
        got, state = gpu_results(dc, inst.reqs.n)
        jobs.append((inst, got, state, "batched inst %d (k=%d)" % (i, inst.k), None))
    # largest data centers first: they set the pool's makespan
    jobs.sort(key=lambda j: -j[0].k)
    errs = compare_chains(jobs)
    assert not errs, "%d data centers differ; first: %s" % (len(errs), errs[0])
    for i in range(0, len(dcs), 8):
        _invariants(ds, dcs[i], wl.instances[i])
    for dc in dcs:
        for f in (ds.FREE_CPU, ds.FREE_MEM, ds.LINK_RES):
            assert np.all(dc.state(f) >= 0)
    plan.close()
    for dc in dcs:
        dc.close()

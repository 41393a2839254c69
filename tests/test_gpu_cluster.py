"""Parity of the thread-block-cluster scheduling kernel (one data center
split over 2-16 blocks that combine column statistics and the argmax
through distributed shared memory) with the FP64 oracle, and with the
one-block kernel: placements, allocations, paths, status, pod scores and the
final state bit-exact for every shape.  Needs a GPU."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W
from parity_util import assert_same_result, assert_same_state, check_instance

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


@pytest.fixture
def launch(ds):
    """Sets launch-table entries for one test and removes them afterwards."""
    keys = []

    def set_(inst, block, ncta):
        key = (inst.k, inst.n_criteria, inst.method, inst.pair_rule)
        ds.set_launch(*key, block, ncta)
        keys.append(key)

    yield set_
    for key in keys:
        ds.set_launch(*key, 0, 1)


def _run(ds, stream, launch, inst, block, ncta, max_requests=None):
    launch(inst, block, ncta)
    dc = ds.load_instance(inst, stream=stream, max_requests=max_requests)
    assert ds.get_launch(dc)[:2] == (block, ncta)
    ds.schedule([dc])
    return dc


@pytest.mark.parametrize("k,block,ncta", [(8, 256, 2), (8, 256, 4), (8, 256, 8),
                                          (16, 512, 2), (16, 256, 4), (16, 512, 8),
                                          (16, 256, 16)])
@pytest.mark.parametrize("method", [W.TOPSIS, W.AHP])
def test_cluster_k8_k16(ds, stream, launch, k, block, ncta, method):
    """Pre-loaded k=8 / k=16 fat-trees, 6 criteria, singleton pods."""
    inst = W.k16(k=k, n_requests=40 if k == 8 else 25, method=method).instances[0]
    dc = _run(ds, stream, launch, inst, block, ncta)
    check_instance(dc, inst, where="cluster k%d %dx%d m%d" % (k, ncta, block, method))


@pytest.mark.parametrize("scheme", ["flat", "clustering", "network"])
def test_cluster_pods_and_intervals(ds, stream, launch, scheme):
    """Multi-container pods with intra-pod links, [min, max] intervals, heavy
    link contention (k=8, 2 blocks per data center), 4 criteria."""
    rng = np.random.Generator(np.random.PCG64(70))
    reqs = [W.gen_request(rng, int(rng.integers(2, 14)), p_edge=0.5,
                          bw=lambda r, m: r.integers(10, 400, m), max_pod=4, intervals=True,
                          intra_pod_links=True) for _ in range(40)]
    inst = W.Instance(8, 16, 32, 1000, 4, W.TOPSIS, W.RATIO, W.WEIGHTS[4][scheme],
                      None, None, None, W.pack_requests(reqs))
    dc = _run(ds, stream, launch, inst, 256, 2)
    check_instance(dc, inst, where="cluster pods %s" % scheme)


@pytest.mark.parametrize("block,ncta", [(512, 2), (512, 4), (256, 8), (1024, 16)])
def test_cluster_k32(ds, stream, launch, block, ncta):
    inst = W.batched(n_instances=1, n_requests=6, ks=(32,), size_hi=48).instances[0]
    dc = _run(ds, stream, launch, inst, block, ncta)
    check_instance(dc, inst, where="cluster k32 %dx%d" % (ncta, block))


@pytest.mark.parametrize("ncta", [4, 8, 16])
@pytest.mark.parametrize("method", [W.TOPSIS, W.AHP])
def test_cluster_k48(ds, stream, launch, ncta, method):
    """The paper-scale fat-tree (27,648 hosts) split over 4-16 blocks."""
    inst = W.k48(n_requests=3, method=method).instances[0]
    dc = _run(ds, stream, launch, inst, 1024, ncta)
    check_instance(dc, inst, where="cluster k48 %d m%d" % (ncta, method))


def test_cluster_releases_across_launches(ds, stream, launch):
    """Schedules and departures over several launches on a cluster-shaped
    data center: FCFS state carried across launches."""
    inst = W.serving(n_instances=2, rate_per_s=400, duration_s=0.5, k=8, size_hi=40,
                     mean_life=5).instances[0]
    launch(inst, 256, 4)
    dc = ds.DataCenter.from_instance(inst, stream=stream)
    odc = O.OracleDC.from_instance(inst)
    results = {}
    step = 0
    for kind, r in inst.ops:
        q = inst.reqs.request(r)
        if kind == 0:
            assert dc.submit(q) == r
            results[r] = odc.schedule(q)
        else:
            dc.release(r)
            if results[r]["status"] == O.ACCEPTED:
                odc.release(q, results[r])
        step += 1
        if step % 9 == 0:
            ds.schedule([dc])
    ds.schedule([dc])
    for r, exp in results.items():
        assert_same_result(dc.query(r), exp, "cluster serving req %d" % r)
    assert_same_state(dc, odc, "cluster serving")


def test_cluster_mixed_plan_matches_one_block(ds, stream, launch):
    """A batched plan mixing cluster shapes (k=16 over 4 blocks, k=8 over 2)
    and one-block data centers (k=4) gives the results of the one-block
    kernel, replayed from a CUDA graph."""
    wl = W.batched(n_instances=6, n_requests=8, ks=(4, 8, 16), size_hi=40)
    ref = []
    for inst in wl.instances:
        dc = ds.load_instance(inst, stream=stream)
        ds.schedule([dc])
        ref.append([dc.query(r) for r in range(inst.reqs.n)])
    launch(wl.instances[1], 256, 2)
    launch(wl.instances[2], 512, 4)
    dcs = [ds.load_instance(inst, stream=stream) for inst in wl.instances]
    assert [ds.get_launch(d)[1] for d in dcs[:3]] == [1, 2, 4]
    plan = ds.Plan(dcs, ds.PLAN_GRAPH | ds.PLAN_RESET)
    for rep in range(2):
        plan.launch(stream)
        plan.collect()
        for i, (dc, inst) in enumerate(zip(dcs, wl.instances)):
            for r in range(inst.reqs.n):
                assert_same_result(dc.query(r), ref[i][r], "mixed %d/%d rep %d" % (i, r, rep))
    for dc, inst in zip(dcs, wl.instances):
        check_instance(dc, inst, where="mixed plan")


def test_cluster_shape_validation(ds):
    """Shapes that cannot hold the data center are refused."""
    with pytest.raises(ds.DcError):
        ds.set_launch(16, 6, W.TOPSIS, W.RATIO, 256, 3)  # 3 does not divide k
    ds.set_launch(16, 6, W.AHP, W.DIFF, 256, 2)  # AHP DIFF runs on clusters too
    ds.set_launch(16, 6, W.AHP, W.DIFF, 0, 1)
    with pytest.raises(ds.DcError):
        ds.set_launch(48, 6, W.TOPSIS, W.RATIO, 512, 8)  # 27,648 hosts > 32 x 512
    with pytest.raises(ds.DcError):
        ds.set_launch(16, 6, W.TOPSIS, W.RATIO, 128, 2)  # cluster blocks are >= 256
    ds.set_launch(16, 6, W.TOPSIS, W.RATIO, 256, 4)
    ds.set_launch(16, 6, W.TOPSIS, W.RATIO, 0, 1)


def test_autotune_keeps_state_and_results(ds, stream):
    """The autotuner times candidate shapes on the queued work of a mixed
    batch, records one shape per kind, and leaves state and queues as they
    were: scheduling afterwards gives the oracle's results, including for an
    instance that already ran a launch before tuning."""
    wl = W.batched(n_instances=4, n_requests=10, ks=(8, 32), size_hi=40)
    dcs = [ds.load_instance(inst, stream=stream, max_requests=4) for inst in wl.instances[:2]]
    ds.schedule(dcs)  # a first launch: 4 requests each
    for dc, inst in zip(dcs, wl.instances[:2]):
        for r in range(4, inst.reqs.n):
            dc.submit(inst.reqs.request(r))
    dcs += [ds.load_instance(inst, stream=stream) for inst in wl.instances[2:]]
    try:
        ent = ds.autotune(dcs, max_ops=6)
        assert len(ent) == 2
        for e in ent:
            assert e["trials"] >= 1 and e["ms"] > 0 and e["ms"] <= e["ms0"] * 1.001
            shape = (e["block"], e["ncta"])
            for dc, inst in zip(dcs, wl.instances):
                if inst.k == e["k"]:
                    assert ds.get_launch(dc)[:2] == shape
        ds.schedule(dcs)
        for dc, inst in zip(dcs, wl.instances):
            check_instance(dc, inst, where="after autotune k%d" % inst.k)
    finally:
        for inst in wl.instances[1:3]:
            ds.set_launch(inst.k, inst.n_criteria, inst.method, inst.pair_rule, 0, 1)


@pytest.mark.parametrize("k,block,ncta", [(8, 256, 2), (16, 256, 4), (16, 512, 8)])
def test_cluster_ahp_diff(ds, stream, launch, k, block, ncta):
    """AHP with the difference rule over a cluster: the histograms, the
    distinct-value lists and their prefix sums are split between the blocks
    (offsets through distributed shared memory), the column and row sums
    between all warps of the cluster."""
    inst = W.k16(k=k, n_requests=30 if k == 8 else 15, method=W.AHP, pair_rule=W.DIFF).instances[0]
    dc = _run(ds, stream, launch, inst, block, ncta)
    check_instance(dc, inst, where="cluster diff k%d %dx%d" % (k, ncta, block))


def test_k48_ahp_diff(ds, stream, launch):
    """AHP DIFF on the paper-scale fat-tree (k = 48, 27,648 hosts) with the
    k48 workload's requests (pods of 1-8, Pareto bandwidths) and 1 Gbps
    links (pre-load scaled from the workload's 40 Gbps one), so that the
    oracle's plain sums over all pairs of the ~1,000 distinct bandwidth
    values stay fast: one block and clusters of 4 and 16 blocks against one
    oracle run, every request and the final state."""
    import dataclasses

    from parity_util import gpu_results

    base = W.k48(n_requests=4, method=W.AHP, pair_rule=W.DIFF).instances[0]
    pre_link = (base.pre_link.astype(np.int64) * 1000 // 40000).astype(np.int32)
    inst = dataclasses.replace(base, link_mbps=1000, pre_link=pre_link)
    runs = []
    for block, ncta in ((1024, 1), (1024, 16), (1024, 4)):
        dc = _run(ds, stream, launch, inst, block, ncta)
        runs.append(((block, ncta),) + gpu_results(dc, inst.reqs.n))
        dc.close()
    ref, odc = O.run_instance(inst)
    assert sum(r["status"] == O.ACCEPTED for r in ref) >= 1
    for shape, got, state in runs:
        for r in range(len(ref)):
            assert_same_result(got[r], ref[r], "k48 diff %s req %d" % (shape, r))
        for f, g in state.items():
            assert np.array_equal(g, odc.state(f)), ("k48 diff state", shape, f)

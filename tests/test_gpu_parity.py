"""Parity of the CUDA path with the FP64 oracle, element by element, on
seeded synthetic workloads: placements, allocations, paths, status and the
integer state bit-exact; certified FP64 pod scores bit-exact; FP32 fast-path
scores within 1e-6 relative.  Needs a GPU."""
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


METHODS = [(W.TOPSIS, W.RATIO), (W.AHP, W.RATIO), (W.AHP, W.DIFF)]


@pytest.mark.parametrize("method,rule", METHODS)
@pytest.mark.parametrize("scheme", ["flat", "clustering", "network"])
def test_small_config(ds, stream, method, rule, scheme):
    inst = W.small(method=method, pair_rule=rule, scheme=scheme).instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    check_instance(dc, inst, where="small/%d/%d/%s" % (method, rule, scheme))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_small_intervals_and_pods(ds, stream, seed):
    rng = np.random.Generator(np.random.PCG64(50 + seed))
    reqs = [W.gen_request(rng, int(rng.integers(2, 12)), p_edge=0.5,
                          bw=lambda r, m: r.integers(10, 400, m), max_pod=3, intervals=True,
                          intra_pod_links=True) for _ in range(40)]
    for method, rule in METHODS:
        inst = W.Instance(4, 16, 32, 1000, 6, method, rule, W.WEIGHTS[6]["network"],
                          None, None, None, W.pack_requests(reqs))
        dc = ds.load_instance(inst, stream=stream)
        ds.schedule([dc])
        check_instance(dc, inst, where="pods/%d/%d/%d" % (seed, method, rule))


@pytest.mark.parametrize("k,n_req", [(8, 120), (16, 60)])
@pytest.mark.parametrize("method,rule", METHODS)
def test_k16_prefix(ds, stream, k, n_req, method, rule):
    inst = W.k16(k=k, n_requests=n_req, method=method, pair_rule=rule).instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    check_instance(dc, inst, where="k%d/%d/%d" % (k, method, rule))


def test_k32_single_block(ds, stream):
    """Largest fat-tree held by one block (8,192 hosts, ~200 KB of shared
    memory), with contention on links."""
    inst = W.batched(n_instances=1, n_requests=6, ks=(32,), size_hi=48).instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    check_instance(dc, inst, where="k32")


def test_incremental_schedules_and_releases(ds, stream):
    """Submit / schedule / release in several launches; FCFS state carried
    across launches."""
    inst = W.serving(n_instances=2, rate_per_s=400, duration_s=0.5, k=8, size_hi=40,
                     mean_life=5).instances[0]
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
        if step % 7 == 0:
            ds.schedule([dc], ds.SCHED_ASYNC if step % 14 == 0 else ds.SCHED_SYNC)
    ds.schedule([dc])
    for r, exp in results.items():
        assert_same_result(dc.query(r), exp, "serving req %d" % r)
    assert_same_state(dc, odc, "serving")


def test_batched_mixed_sizes_match_alone(ds, stream):
    """Instances of different sizes in one batched launch give the same
    results as each instance scheduled alone, and as the oracle."""
    wl = W.batched(n_instances=6, n_requests=8, ks=(4, 8, 16), size_hi=40)
    dcs = [ds.load_instance(inst, stream=stream) for inst in wl.instances]
    ds.schedule(dcs)
    for i, (dc, inst) in enumerate(zip(dcs, wl.instances)):
        check_instance(dc, inst, where="batch inst %d" % i)
        alone = ds.load_instance(inst, stream=stream)
        ds.schedule([alone])
        for r in range(inst.reqs.n):
            assert_same_result(alone.query(r), dc.query(r), "alone vs mix %d/%d" % (i, r))


def test_plan_graph_replay(ds, stream):
    """A captured plan replayed with a state reset gives identical results."""
    wl = W.batched(n_instances=4, n_requests=6, ks=(8, 16), size_hi=30)
    dcs = [ds.load_instance(inst, stream=stream) for inst in wl.instances]
    plan = ds.Plan(dcs, ds.PLAN_GRAPH | ds.PLAN_RESET)
    first = None
    for rep in range(3):
        plan.launch(stream)
        plan.collect()
        dec, hr, nk, t0 = plan.stats()
        assert dec > 0 and hr >= dec * 128 and nk == 2
        now = [[dc.query(r) for r in range(inst.reqs.n)] for dc, inst in zip(dcs, wl.instances)]
        if first is None:
            first = now
        else:
            for a, b in zip(first, now):
                for x, y in zip(a, b):
                    assert_same_result(x, y, "replay %d" % rep)
    for dc, inst in zip(dcs, wl.instances):
        check_instance(dc, inst, where="plan")


@pytest.mark.parametrize("method,rule", METHODS)
def test_rank_hosts_scores(ds, stream, method, rule):
    """Per-host viability and criteria exact, FP64 scores bit-exact, FP32
    scores within 1e-6 relative of the oracle, for pods with placed
    neighbours on a pre-loaded k=16 fat-tree."""
    inst = W.k16(n_requests=20, method=method, pair_rule=rule).instances[0]
    dc = ds.DataCenter.from_instance(inst, stream=stream)
    odc = O.OracleDC.from_instance(inst)
    rng = np.random.default_rng(7)
    for r in range(8):
        q = inst.reqs.request(r)
        P = int(q["pod"].max()) + 1
        host_of = rng.integers(0, dc.H, len(q["pod"])).astype(np.int32)
        for g in sorted(set([0, P // 2, P - 1])):
            ho = host_of.copy()
            ho[q["pod"] >= g] = -1
            feas, s32, s64, crit, nv = dc.rank_hosts(q, g, ho)
            of, oc, osc = odc.rank_pod(q, g, ho)
            assert np.array_equal(feas, of)
            assert nv == int(of.sum())
            assert np.array_equal(crit[of], oc[of].astype(np.int32))
            assert np.array_equal(s64[of], osc[of])
            rel = np.abs(s32[of].astype(np.float64) - osc[of]) / np.maximum(osc[of].max(), 1e-300)
            assert rel.max(initial=0) < 1e-6, rel.max()
            assert np.all(np.isnan(s32[~of])) and np.all(np.isnan(s64[~of]))


def test_full_k16_whole_chain(ds, stream):
    """The full 1,000-request k=16 workload (1,024 hosts, 0-70 % pre-load,
    4-64 containers, 6 criteria, TOPSIS) in one launch: every request and
    the final state element by element against the oracle."""
    inst = W.k16().instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    ref = check_instance(dc, inst, where="k16 full")
    assert len(ref) == 1000
    n_acc = sum(r["status"] == O.ACCEPTED for r in ref)
    assert 0 < n_acc < 1000  # the late requests meet a full data center


@pytest.mark.parametrize("method,rule,n_req", [(W.TOPSIS, W.RATIO, 40), (W.AHP, W.RATIO, 20)])
def test_k48_chain_launch_shapes(ds, stream, method, rule, n_req):
    """The paper-scale fat-tree (k = 48, 27,648 hosts, state in L2-resident
    global memory): the first n_req requests of the 200-request workload
    (pods of 1-8 containers, Pareto bandwidths, 0-100 % pre-load), one
    block and thread-block clusters of 4, 8 and 16 blocks of 1024 threads (the shapes the
    benchmark's autotuner chooses among), every request and the final state
    element by element against one oracle run."""
    from parity_util import compare_chain, gpu_results

    inst = W.k48(n_requests=n_req, method=method, pair_rule=rule).instances[0]
    key = (inst.k, inst.n_criteria, inst.method, inst.pair_rule)
    runs = []
    for block, ncta in ((1024, 1), (1024, 16), (1024, 8), (1024, 4)):
        ds.set_launch(*key, block, ncta)
        try:
            dc = ds.load_instance(inst, stream=stream)
            ds.schedule([dc])
            runs.append(((block, ncta),) + gpu_results(dc, inst.reqs.n))
            dc.close()
        finally:
            ds.set_launch(*key, 0, 1)
    ref, odc = O.run_instance(inst)
    assert sum(r["n_decisions"] for r in ref) > 20 * n_req
    for shape, got, state in runs:
        for r in range(len(ref)):
            assert_same_result(got[r], ref[r], "k48 %s req %d" % (shape, r))
        for f, g in state.items():
            assert np.array_equal(g, odc.state(f)), ("k48 state", shape, f)


def test_invalid_inputs_rejected(ds, stream):
    dc = ds.DataCenter(4, 32, 64, 1000, 4, ds.TOPSIS, ds.RATIO, (0.25,) * 4, stream=stream)
    good = W.gen_request(np.random.default_rng(0), 3, p_edge=1.0,
                         bw=lambda r, m: r.integers(1, 5, m))
    for bad in (dict(good, pod=np.array([0, 2, 2], np.int32)),
                dict(good, dst=good["src"].copy()),
                dict(good, cpu_min=good["cpu_max"] + 1)):
        with pytest.raises(ds.DcError):
            dc.submit(bad)
    with pytest.raises(ds.DcError):
        ds.DataCenter(5, 32, 64, 1000, 4, ds.TOPSIS, ds.RATIO, (0.25,) * 4)
    with pytest.raises(ds.DcError):
        ds.DataCenter(4, 32, 64, 1000, 4, ds.TOPSIS, ds.RATIO, (0.25,) * 4,
                      pre_cpu=np.full(16, 40, np.int32))
    with pytest.raises(ds.DcError):
        dc.release(99)

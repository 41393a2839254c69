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
    if rule == W.DIFF:
        n_req = n_req // 4  # O(F^2) per criterion and decision in both implementations
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


@pytest.mark.parametrize("method,rule", [(W.TOPSIS, W.RATIO), (W.AHP, W.RATIO)])
def test_k48_global_state(ds, stream, method, rule):
    """k = 48 (27,648 hosts, the paper-scale fat-tree): the state lives in an
    L2-resident global copy instead of shared memory.  Pods of 1-8
    containers, intra-pod links, Pareto bandwidths, 0-100 % pre-load."""
    inst = W.k48(n_requests=3, method=method, pair_rule=rule).instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    check_instance(dc, inst, where="k48/%d" % method)


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


def test_full_k16_sampled(ds, stream):
    """The full 1,000-request k=16 workload in the benchmark's launch
    configuration: every request checked against invariants (capacity never
    exceeded, conservation, path validity) and the first 150 requests
    element by element against the oracle."""
    inst = W.k16().instances[0]
    dc = ds.load_instance(inst, stream=stream)
    ds.schedule([dc])
    ref = check_instance_prefix(dc, inst, 150)
    H = inst.hosts
    used_c = np.zeros(H, np.int64)
    used_m = np.zeros(H, np.int64)
    used_l = np.zeros(3 * H, np.int64)
    for r in range(inst.reqs.n):
        out = dc.query(r)
        q = inst.reqs.request(r)
        if out["status"] == ds.ACCEPTED:
            np.add.at(used_c, out["host"], out["cpu"])
            np.add.at(used_m, out["host"], out["mem"])
            assert np.all((out["cpu"] >= q["cpu_min"]) & (out["cpu"] <= q["cpu_max"]))
            for e in range(len(q["src"])):
                links = out["path"][6 * e:6 * e + 6]
                np.add.at(used_l, links[links >= 0], out["bw"][e])
        else:
            assert np.all(out["host"] == -1)
    cap_c = 32 - (inst.pre_cpu.astype(np.int64))
    cap_m = 64 - (inst.pre_mem.astype(np.int64))
    assert np.array_equal(dc.state(ds.FREE_CPU), cap_c - used_c)
    assert np.array_equal(dc.state(ds.FREE_MEM), cap_m - used_m)
    assert np.array_equal(dc.state(ds.LINK_RES), 10000 - inst.pre_link.astype(np.int64) - used_l)
    assert np.all(dc.state(ds.LINK_RES) >= 0) and np.all(dc.state(ds.FREE_CPU) >= 0)


def check_instance_prefix(dc, inst, n):
    ref, _ = O.run_instance(inst, max_requests=n)
    for r in range(n):
        assert_same_result(dc.query(r), ref[r], "k16 full, req %d" % r)
    return ref


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

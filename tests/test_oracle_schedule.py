"""Pins of the oracle's criteria, viability, commit and greedy FCFS loop:
brute force over the networkx fat-tree, the MILP constraints of Eqs. 4-8
checked by oracle/milp_brute.py on every accepted request, resource
conservation, rollback and release.  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W


def _random_state(rng, k, cap_cpu=32, cap_mem=64, link=1000, levels=None):
    H = k ** 3 // 4
    pre_cpu = rng.integers(0, cap_cpu + 1, H).astype(np.int32)
    pre_mem = rng.integers(0, cap_mem + 1, H).astype(np.int32)
    if levels:
        pre_link = (link - rng.integers(0, levels, 3 * H) * (link // levels)).astype(np.int32)
    else:
        pre_link = rng.integers(0, link + 1, 3 * H).astype(np.int32)
    pre_cpu[rng.random(H) < 0.3] = 0
    pre_mem[pre_cpu == 0] = 0
    return pre_cpu, pre_mem, pre_link


@pytest.mark.parametrize("seed", range(6))
def test_criteria_and_viability_bruteforce(seed):
    """c0..c5 and viability of every host for a pod with placed neighbours,
    recomputed from their definitions with networkx shortest paths."""
    pytest.importorskip("networkx")
    from fattree_ref import build, widest_shortest

    rng = np.random.default_rng(seed)
    k = 4 if seed < 4 else 6
    H = k ** 3 // 4
    G, lid = build(k)
    link = 1000
    pc, pm, pl = _random_state(rng, k, link=link, levels=4 if seed % 2 else None)
    dc = O.OracleDC(k, 32, 64, link, 6, O.TOPSIS, O.RATIO, (1 / 6,) * 6, pc, pm, pl)
    res = dc.state(O.LINK_RES)
    free_cpu, free_mem = dc.state(O.FREE_CPU), dc.state(O.FREE_MEM)
    ctr, pre = dc.state(O.CTR), dc.state(O.PRE)
    n = 7
    q = W.gen_request(rng, n, p_edge=0.5, bw=lambda r, m: r.integers(0, 400, m))
    g = n - 1  # last pod; every other pod placed on random hosts
    host_of = rng.integers(0, H, n).astype(np.int32)
    host_of[g] = -1
    if seed == 0:
        host_of[:g] = 3  # neighbours stacked on one host
    feas, crit, score = dc.rank_pod(q, g, host_of)

    pe = [(e, int(host_of[q["dst"][e] if q["src"][e] == g else q["src"][e]]))
          for e in range(len(q["src"])) if g in (q["src"][e], q["dst"][e])]
    need = {}
    for e, v in pe:
        need[v] = max(need.get(v, -1), int(q["bw_min"][e]))
    for u in range(H):
        bott = {v: (link if v == u else widest_shortest(G, lid, res, u, v)[0]) for v in need}
        c4 = min(bott.values()) if pe else res[u]
        hops = {v: (0 if v == u else widest_shortest(G, lid, res, u, v)[2]) for v in need}
        c5 = sum(6 - hops[v] for _, v in pe)
        exp = [free_cpu[u], free_mem[u], int(ctr[u] > 0 or pre[u] > 0), res[u], c4, c5]
        assert list(crit[u]) == exp, u
        ok = (free_cpu[u] >= q["cpu_min"][g] and free_mem[u] >= q["mem_min"][g]
              and all(bott[v] >= need[v] for v in need if v != u))
        assert feas[u] == ok, u
    # scores of viable hosts are TOPSIS over the viable rows
    F = np.nonzero(feas)[0]
    if len(F):
        assert np.array_equal(score[F], O.topsis(crit[F], (1 / 6,) * 6))
        assert np.all(np.isnan(score[~feas]))


def _check_run(inst, n_req):
    pytest.importorskip("networkx")
    from fattree_ref import build
    from oracle.milp_brute import check_placement

    G, lid = build(inst.k)
    dc = O.OracleDC.from_instance(inst)
    H = inst.hosts
    cpu0, mem0, res0 = dc.state(O.FREE_CPU), dc.state(O.FREE_MEM), dc.state(O.LINK_RES)
    used_cpu = np.zeros(H, np.int64)
    used_mem = np.zeros(H, np.int64)
    used_link = np.zeros(3 * H, np.int64)
    results = []
    n_acc = 0
    for r in range(n_req):
        q = inst.reqs.request(r)
        fc, fm, rs = dc.state(O.FREE_CPU), dc.state(O.FREE_MEM), dc.state(O.LINK_RES)
        out = dc.schedule(q)
        results.append((q, out))
        if out["status"] == O.ACCEPTED:
            n_acc += 1
            assert check_placement(G, lid, fc, fm, rs, q, out) == []
            assert np.all(out["pod_score"] >= 0)
            for i, u in enumerate(out["host"]):
                used_cpu[u] += out["cpu"][i]
                used_mem[u] += out["mem"][i]
            for e in range(len(q["src"])):
                for x in out["path"][6 * e:6 * e + 6]:
                    if x >= 0:
                        used_link[x] += out["bw"][e]
        else:
            assert out["status"] == O.REJECTED
            assert np.all(out["host"] == -1) and np.all(out["bw"] == 0)
            assert np.all(out["path"] == -1)
            # rollback leaves no residue
            assert np.array_equal(dc.state(O.FREE_CPU), fc)
            assert np.array_equal(dc.state(O.FREE_MEM), fm)
            assert np.array_equal(dc.state(O.LINK_RES), rs)
        assert out["n_decisions"] >= 1 or len(q["pod"]) == 0
        # conservation
        assert np.array_equal(cpu0 - used_cpu, dc.state(O.FREE_CPU))
        assert np.array_equal(mem0 - used_mem, dc.state(O.FREE_MEM))
        assert np.array_equal(res0 - used_link, dc.state(O.LINK_RES))
        assert np.all(dc.state(O.LINK_RES) >= 0)
    # releasing everything restores the initial state
    for q, out in results:
        if out["status"] == O.ACCEPTED:
            dc.release(q, out)
    assert np.array_equal(dc.state(O.FREE_CPU), cpu0)
    assert np.array_equal(dc.state(O.FREE_MEM), mem0)
    assert np.array_equal(dc.state(O.LINK_RES), res0)
    assert np.all(dc.state(O.CTR) == 0)
    return n_acc


@pytest.mark.parametrize("method,rule", [(O.TOPSIS, O.RATIO), (O.AHP, O.RATIO), (O.AHP, O.DIFF)])
@pytest.mark.parametrize("scheme", ["flat", "clustering", "network"])
def test_small_config_feasible_and_conserving(method, rule, scheme):
    wl = W.small(method=method, pair_rule=rule, scheme=scheme)
    n_acc = _check_run(wl.instances[0], 10)
    assert n_acc >= 1


def test_small_intervals_and_pods():
    """[min, max] intervals (Eqs. 6-7), pods of several containers and
    intra-pod links on a k=4 fat-tree."""
    rng = np.random.Generator(np.random.PCG64(11))
    reqs = [W.gen_request(rng, int(rng.integers(2, 9)), p_edge=0.5,
                          bw=lambda r, m: r.integers(10, 300, m), max_pod=3, intervals=True,
                          intra_pod_links=True) for _ in range(25)]
    inst = W.Instance(4, 16, 32, 1000, 6, O.TOPSIS, O.RATIO, W.WEIGHTS[6]["network"],
                      None, None, None, W.pack_requests(reqs))
    assert _check_run(inst, 25) >= 1


def test_k8_prefix_feasible():
    wl = W.k16(k=8, n_requests=40)
    _check_run(wl.instances[0], 40)


def test_greedy_vs_exhaustive_tiny():
    """Every accepted placement is feasible (asserted by _check_run); for a
    rejected request the exhaustive search reports whether the MILP could
    have placed it (greedy is a heuristic: reported, not asserted), and any
    request the search proves infeasible must be rejected."""
    pytest.importorskip("networkx")
    from fattree_ref import build
    from oracle.milp_brute import exhaustive_feasible

    G, lid = build(4)
    rng = np.random.Generator(np.random.PCG64(12))
    dc = O.OracleDC(4, 8, 16, 300, 4, O.TOPSIS, O.RATIO, W.WEIGHTS[4]["network"])
    missed = 0
    for r in range(30):
        q = W.gen_request(rng, int(rng.integers(2, 4)), p_edge=0.6,
                          bw=lambda r_, m: r_.integers(50, 250, m), cpu_hi=4, mem_hi=8)
        fc, fm, rs = dc.state(O.FREE_CPU), dc.state(O.FREE_MEM), dc.state(O.LINK_RES)
        out = dc.schedule(q)
        feasible = exhaustive_feasible(G, lid, fc, fm, rs, q)
        if feasible is False:
            assert out["status"] == O.REJECTED
        if out["status"] == O.REJECTED and feasible:
            missed += 1
    print("requests the exhaustive MILP search could place but greedy rejected:", missed)


def test_release_and_reschedule_same_result():
    wl = W.small(n_requests=6)
    inst = wl.instances[0]
    dc = O.OracleDC.from_instance(inst)
    first = [dc.schedule(inst.reqs.request(r)) for r in range(6)]
    for r in range(6):
        if first[r]["status"] == O.ACCEPTED:
            dc.release(inst.reqs.request(r), first[r])
    again = [dc.schedule(inst.reqs.request(r)) for r in range(6)]
    for a, b in zip(first, again):
        for key in ("host", "cpu", "mem", "bw", "path", "pod_score"):
            assert np.array_equal(a[key], b[key])


def test_invalid_requests_rejected_by_validation():
    dc = O.OracleDC(4, 32, 64, 1000, 4, O.TOPSIS, O.RATIO, (0.25,) * 4)
    good = W.gen_request(np.random.default_rng(0), 3, p_edge=1.0, bw=lambda r, m: r.integers(1, 5, m))
    bad_pod = dict(good, pod=np.array([0, 2, 2], np.int32))        # pod ids not dense
    bad_loop = dict(good, dst=good["src"].copy())                   # src == dst
    bad_int = dict(good, cpu_min=good["cpu_max"] + 1)               # min > max
    for q in (bad_pod, bad_loop, bad_int):
        with pytest.raises(ValueError):
            dc.schedule(q)

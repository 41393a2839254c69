"""Pins of the oracle's utilities (Sec. II-B, Eqs. 1-2) and fragmentation
(Sec. II-B) against hand-worked placements and against counts taken
independently from the placements themselves."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W


def _req(cpu, mem, src=(), dst=(), bw=(), pod=None):
    n = len(cpu)
    return {
        "cpu_min": np.array([c[0] for c in cpu], np.int32),
        "cpu_max": np.array([c[1] for c in cpu], np.int32),
        "mem_min": np.array([m[0] for m in mem], np.int32),
        "mem_max": np.array([m[1] for m in mem], np.int32),
        "pod": np.array(pod if pod is not None else range(n), np.int32),
        "src": np.array(src, np.int32), "dst": np.array(dst, np.int32),
        "bw_min": np.array([b[0] for b in bw], np.int32),
        "bw_max": np.array([b[1] for b in bw], np.int32),
    }


def _dc(k=4, cpu=32, mem=64, mbps=1000, pre_cpu=None, pre_mem=None, pre_link=None):
    return O.OracleDC(k, cpu, mem, mbps, 4, O.TOPSIS, O.RATIO, [0.25] * 4, pre_cpu, pre_mem,
                      pre_link)


def test_max_allocation_gives_utility_one():
    """Room for every maximum: the commit takes the maxima, U = 1 (the
    paper's optimum)."""
    dc = _dc()
    q = _req([(1, 4), (2, 3)], [(2, 8), (1, 5)], src=[0], dst=[1], bw=[(10, 100)])
    out = dc.schedule(q)
    assert out["status"] == O.ACCEPTED
    uc, ue = O.utilities(q, out)
    assert list(uc) == [1.0, 1.0] and list(ue) == [1.0]


def test_minimum_allocation_hand_worked():
    """Every host pre-loaded to 2 free CPU units: a container asking CPU
    [1, 4] and memory [2, 8] gets CPU 1 (the maximum does not fit) and memory
    8, so U = (1/4 + 8/8) / 2 = 0.625.  Every link of the fat-tree carries at
    most 50 Mbps, so a link asking [10, 100] Mbps gets its minimum: U = 0.1."""
    H = 16
    dc = _dc(mbps=1000, pre_cpu=np.full(H, 30, np.int32),
             pre_link=np.full(3 * H, 950, np.int32))
    q = _req([(1, 4), (1, 1)], [(2, 8), (1, 1)], src=[0], dst=[1], bw=[(10, 100)])
    out = dc.schedule(q)
    assert out["status"] == O.ACCEPTED
    uc, ue = O.utilities(q, out)
    assert uc[0] == 0.625 and uc[1] == 1.0
    if out["host"][0] != out["host"][1]:
        assert out["bw"][0] == 10 and ue[0] == 0.1
    else:  # both on one host: no network link, bw_max
        assert ue[0] == 1.0


def test_rejected_request_has_zero_utilities():
    dc = _dc(k=2)  # 2 hosts of 32 CPU
    q = _req([(20, 20)] * 4, [(1, 1)] * 4)
    out = dc.schedule(q)
    assert out["status"] == O.REJECTED
    uc, ue = O.utilities(q, out)
    assert np.all(uc == 0.0)


def test_zero_maximum_counts_as_satisfied():
    dc = _dc()
    q = _req([(0, 0)], [(1, 2)])
    out = dc.schedule(q)
    uc, _ = O.utilities(q, out)
    assert uc[0] == (1.0 + 1.0) / 2.0


def _independent_counts(dc, results, reqs, pre_hosts, pre_links):
    """Active servers and links counted from the placements themselves."""
    hosts = set(pre_hosts)
    links = set(pre_links)
    for q, out in zip(reqs, results):
        if out["status"] != O.ACCEPTED:
            continue
        hosts.update(int(h) for h in out["host"])
        for e in range(len(q["src"])):
            if out["bw"][e] > 0:
                links.update(int(l) for l in out["path"][6 * e:6 * e + 6] if l >= 0)
    return len(hosts), len(links)


def test_fragmentation_empty_and_full():
    dc = _dc()
    a, b, fs, fl = dc.fragmentation()
    assert (a, b, fs, fl) == (0, 0, 0.0, 0.0)
    H = 16
    dc = _dc(pre_cpu=np.ones(H, np.int32), pre_link=np.ones(3 * H, np.int32))
    a, b, fs, fl = dc.fragmentation()
    assert (a, b, fs, fl) == (H, 3 * H, 1.0, 1.0)


@pytest.mark.parametrize("seed", [0, 1])
def test_fragmentation_matches_placements(seed):
    """F(N^s) and F(E^s) after a k=8 workload with partial pre-load equal
    the counts taken from the placements (hosts used, links on reserved
    paths) plus the pre-loaded ones; releases bring them back."""
    inst = W.k16(seed=seed, k=8, n_requests=30).instances[0]
    dc = O.OracleDC.from_instance(inst)
    pre_hosts = [h for h in range(inst.hosts) if inst.pre_cpu[h] > 0 or inst.pre_mem[h] > 0]
    pre_links = [l for l in range(3 * inst.hosts) if inst.pre_link[l] > 0]
    reqs = [inst.reqs.request(r) for r in range(inst.reqs.n)]
    results = [dc.schedule(q) for q in reqs]
    a, b, fs, fl = dc.fragmentation()
    ea, eb = _independent_counts(dc, results, reqs, pre_hosts, pre_links)
    assert (a, b) == (ea, eb)
    assert fs == ea / inst.hosts and fl == eb / (3 * inst.hosts)
    for q, out in zip(reqs, results):
        if out["status"] == O.ACCEPTED:
            dc.release(q, out)
    a, b, _, _ = dc.fragmentation()
    assert (a, b) == (len(pre_hosts), len(pre_links))


def test_utilities_of_interval_workload_bounds():
    """Interval requests on a pre-loaded k=8 fat-tree: every utility of an
    accepted request lies in [min/max, 1] per its own bounds."""
    inst = W.k16(seed=3, k=8, n_requests=40, intervals=True).instances[0]
    dc = O.OracleDC.from_instance(inst)
    seen_below_one = False
    for r in range(inst.reqs.n):
        q = inst.reqs.request(r)
        out = dc.schedule(q)
        uc, ue = O.utilities(q, out)
        if out["status"] != O.ACCEPTED:
            assert np.all(uc == 0) and np.all(ue == 0)
            continue
        lo = (q["cpu_min"] / np.maximum(q["cpu_max"], 1) + q["mem_min"] / np.maximum(q["mem_max"], 1)) / 2
        assert np.all(uc >= lo - 1e-15) and np.all(uc <= 1.0)
        lo_e = q["bw_min"] / np.maximum(q["bw_max"], 1)
        assert np.all(ue >= lo_e - 1e-15) and np.all(ue <= 1.0)
        seen_below_one = seen_below_one or bool(np.any(uc < 1.0) or np.any(ue < 1.0))
    assert seen_below_one

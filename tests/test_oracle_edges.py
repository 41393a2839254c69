"""Degenerate requests on the oracle, pinned by the placement constraints
alone: an empty request, a container larger than every host, a pod that fits
no single host although its containers would fit apart (a pod shares one
host), links inside a pod or between containers on one host (no network
link, bw^max), and the smallest fat-tree (k = 2).  CPU only."""
import numpy as np

import oracle as O

Z = np.zeros(0, np.int32)


def _req(cpu, pod=None, src=(), dst=(), bw=(), mem=None):
    n = len(cpu)
    cpu = np.asarray(cpu, np.int32)
    mem = np.ones(n, np.int32) if mem is None else np.asarray(mem, np.int32)
    bw = np.asarray(bw, np.int32)
    return {"cpu_min": cpu, "cpu_max": cpu.copy(), "mem_min": mem, "mem_max": mem.copy(),
            "pod": np.arange(n, dtype=np.int32) if pod is None else np.asarray(pod, np.int32),
            "src": np.asarray(src, np.int32), "dst": np.asarray(dst, np.int32),
            "bw_min": bw, "bw_max": bw.copy()}


def _dc(k=4, host_cpu=8, link=100, pre_cpu=None):
    return O.OracleDC(k, host_cpu, 16, link, 4, O.TOPSIS, O.RATIO, [0.25] * 4, pre_cpu, None,
                      None)


def _snapshot(dc):
    return [dc.state(f).copy() for f in (O.FREE_CPU, O.FREE_MEM, O.CTR, O.LINK_RES)]


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_empty_request_is_accepted_and_changes_nothing():
    dc = _dc()
    before = _snapshot(dc)
    out = dc.schedule({"cpu_min": Z, "cpu_max": Z, "mem_min": Z, "mem_max": Z, "pod": Z,
                       "src": Z, "dst": Z, "bw_min": Z, "bw_max": Z})
    assert out["status"] == O.ACCEPTED and out["n_decisions"] == 0
    assert _same(before, _snapshot(dc))


def test_container_larger_than_every_host_is_rejected():
    dc = _dc(host_cpu=8)
    before = _snapshot(dc)
    out = dc.schedule(_req([9]))
    assert out["status"] == O.REJECTED
    assert np.all(out["host"] == -1) and np.all(out["cpu"] == 0)
    assert _same(before, _snapshot(dc))


def test_pod_shares_one_host():
    """Two 5-CPU containers on 8-CPU hosts: as one pod they fit no host (the
    pod is placed on a single host) and the request is rejected; as two
    singleton pods they are placed on two hosts."""
    dc = _dc(host_cpu=8)
    before = _snapshot(dc)
    assert dc.schedule(_req([5, 5], pod=[0, 0]))["status"] == O.REJECTED
    assert _same(before, _snapshot(dc))
    out = dc.schedule(_req([5, 5]))
    assert out["status"] == O.ACCEPTED and out["host"][0] != out["host"][1]


def test_links_inside_a_pod_use_no_network():
    """A pod of two containers linked to each other: both on one host, the
    link gets bw^max, no path and no link residual changes."""
    dc = _dc()
    link_before = dc.state(O.LINK_RES).copy()
    out = dc.schedule(_req([2, 2], pod=[0, 0], src=[0], dst=[1], bw=[70]))
    assert out["status"] == O.ACCEPTED and out["host"][0] == out["host"][1]
    assert out["bw"][0] == 70 and np.all(out["path"] == -1)
    assert np.array_equal(link_before, dc.state(O.LINK_RES))


def test_link_between_containers_on_one_host_uses_no_network():
    """Singleton pods that can only land on the same host (every other host
    pre-loaded full): their link needs no network link either."""
    H = 16
    pre = np.full(H, 8, np.int32)
    pre[5] = 0
    dc = _dc(host_cpu=8, pre_cpu=pre)
    link_before = dc.state(O.LINK_RES).copy()
    out = dc.schedule(_req([3, 3], src=[0], dst=[1], bw=[90]))
    assert out["status"] == O.ACCEPTED and list(out["host"]) == [5, 5]
    assert out["bw"][0] == 90 and np.all(out["path"] == -1)
    assert np.array_equal(link_before, dc.state(O.LINK_RES))


def test_smallest_fat_tree():
    """k = 2: two hosts, each alone under its edge switch; a link between
    containers on the two hosts crosses host, edge-aggregation and
    aggregation-core links (6 links, bottleneck reserved on each) or, within
    one pod, 4 links."""
    dc = O.OracleDC(2, 4, 8, 100, 4, O.TOPSIS, O.RATIO, [0.25] * 4, None, None, None)
    assert dc.state(O.FREE_CPU).shape == (2,) and dc.state(O.LINK_RES).shape == (6,)
    out = dc.schedule(_req([4, 4], src=[0], dst=[1], bw=[30]))
    assert out["status"] == O.ACCEPTED and sorted(out["host"]) == [0, 1]
    links = out["path"][out["path"] >= 0]
    assert out["bw"][0] == 30 and len(links) in (4, 6) and len(set(links)) == len(links)
    res = dc.state(O.LINK_RES)
    assert np.all(res[links] == 70)
    assert np.all(np.delete(res, links) == 100)

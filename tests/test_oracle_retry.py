"""Pin of the candidate order after a failed commit (Sec. V-C: candidates
"sorted on decreasing order" of their rank, tried one after another), on a
hand-built k=4 fat-tree where the best-ranked hosts cannot carry the pod's
links.  CPU only.

The data center (16 hosts of 32 CPU / 64 memory, 1000 Mbps links):

  host 0       empty; the only host with room for pod 0 (20 CPU)
  hosts 8, 9   free (19 CPU, 57 mem), uplink 978; edge switch 4 has
               aggregation links of residual 100 (a = 0) and 50 (a = 1)
  hosts 4, 12  free (17, 3), uplink 993 (identical twins)
  host 2       free (14, 27), uplink 128
  the rest     10 free CPU: no room for pod 1 (13 CPU)

Request: pod 0 = containers 0, 1 (10 CPU, 1 mem each), pod 1 = container 2
(13 CPU, 1 mem), links 0-2 and 1-2 of exactly 60 Mbps.  Pod 0 can only go to
host 0.  For pod 1 the viable hosts are 2, 4, 8, 9, 12, every one with a
path of bottleneck >= 60 to host 0, and the ranking (TOPSIS, AHP RATIO and
AHP DIFF alike) is 8 = 9 > 4 = 12 > 2.  Hosts 8 and 9 pass the viability
check, yet their commit fails: the first link takes 60 of the a = 0 link of
edge switch 4 (100 -> 40), after which no path to host 0 has 60 left
(max(40, 50) < 60), so the first reservation is undone.  The pod then lands
on host 4.  Each plausible mistake in the retry gives another host:

  scores recomputed over the hosts not yet tried  -> host 2 (the ranking of
      2, 4, 12 alone puts 2 first, checked below with the pinned scorers)
  candidates by host index instead of by score    -> host 2
  ties broken towards the higher index ('>=')     -> host 12
"""
import numpy as np
import pytest

import oracle as O

K, H, CAP_CPU, CAP_MEM, LINK = 4, 16, 32, 64, 1000
W4 = (0.25, 0.25, 0.25, 0.25)

# free (cpu, mem, uplink residual) of the hosts viable for pod 1
VIABLE = {8: (19, 57, 978), 9: (19, 57, 978), 4: (17, 3, 993), 12: (17, 3, 993),
          2: (14, 27, 128)}

METHODS = [(O.TOPSIS, O.RATIO), (O.AHP, O.RATIO), (O.AHP, O.DIFF)]


def _link_ea(e, a):
    return H + e * (K // 2) + a


def _state():
    pre_cpu = np.full(H, CAP_CPU - 10, np.int32)
    pre_mem = np.zeros(H, np.int32)
    pre_link = np.zeros(3 * H, np.int32)
    pre_cpu[0] = 0
    for h, (c, m, up) in VIABLE.items():
        pre_cpu[h] = CAP_CPU - c
        pre_mem[h] = CAP_MEM - m
        pre_link[h] = LINK - up
    pre_link[_link_ea(4, 0)] = LINK - 100
    pre_link[_link_ea(4, 1)] = LINK - 50
    return pre_cpu, pre_mem, pre_link


def _request(cpu_pod1=13):
    i32 = lambda *v: np.array(v, np.int32)  # noqa: E731
    return {"cpu_min": i32(10, 10, cpu_pod1), "cpu_max": i32(10, 10, cpu_pod1),
            "mem_min": i32(1, 1, 1), "mem_max": i32(1, 1, 1), "pod": i32(0, 0, 1),
            "src": i32(0, 1), "dst": i32(2, 2), "bw_min": i32(60, 60), "bw_max": i32(60, 60)}


def _dc(method, rule):
    pc, pm, pl = _state()
    return O.OracleDC(K, CAP_CPU, CAP_MEM, LINK, 4, method, rule, W4, pc, pm, pl)


def _score(method, rule, X):
    return O.topsis(X, W4) if method == O.TOPSIS else O.ahp(X, W4, rule)


def _rows(hosts):
    # criteria (free CPU, free memory, active flag, uplink): every viable
    # host carries pre-load, so its flag is 1
    return np.array([(VIABLE[h][0], VIABLE[h][1], 1, VIABLE[h][2]) for h in hosts], np.int64)


@pytest.mark.parametrize("method,rule", METHODS)
def test_design_distinguishes_the_wrong_orders(method, rule):
    """The hand-built ranking: 8 = 9 > 4 = 12 > 2 over the five viable
    hosts, while 2, 4, 12 alone rank 2 first; and the oracle's own ranking
    of pod 1 (pod 0 on host 0) is exactly that, host by host."""
    hosts = sorted(VIABLE)
    s = dict(zip(hosts, _score(method, rule, _rows(hosts))))
    assert s[8] == s[9] > s[4] == s[12] > s[2]
    rest = [2, 4, 12]
    s2 = dict(zip(rest, _score(method, rule, _rows(rest))))
    assert s2[2] > s2[4] == s2[12]

    dc = _dc(method, rule)
    host_of = np.array([0, 0, -1], np.int32)
    # the ranking is taken on the state after pod 0's commit
    cpu = dc.state(O.FREE_CPU)
    cpu[0] -= 20
    dc.set_state(O.FREE_CPU, cpu)
    mem = dc.state(O.FREE_MEM)
    mem[0] -= 2
    dc.set_state(O.FREE_MEM, mem)
    feas, crit, score = dc.rank_pod(_request(), 1, host_of)
    assert sorted(np.nonzero(feas)[0].tolist()) == hosts
    assert np.array_equal(crit[hosts], _rows(hosts))
    assert all(score[h] == s[h] for h in hosts)


@pytest.mark.parametrize("method,rule", METHODS)
def test_failed_commits_fall_to_next_in_score_order(method, rule):
    dc = _dc(method, rule)
    res0 = dc.state(O.LINK_RES)
    out = dc.schedule(_request())
    assert out["status"] == O.ACCEPTED
    assert out["n_decisions"] == 2  # one per pod; retries are not decisions
    # 8 and 9 failed (second link), 4 is next; 12 (its twin, higher index)
    # and 2 (first by index, first after a recomputation) are not reached
    assert out["host"].tolist() == [0, 0, 4]
    assert out["cpu"].tolist() == [10, 10, 13] and out["mem"].tolist() == [1, 1, 1]
    # both links take the lowest-index widest path host 0 -> host 4
    # (inter-pod; a = 0, c = 0 on ties: every candidate is capped by the uplinks)
    path = [0, _link_ea(0, 0), 2 * H + 0, 2 * H + (1 * 2 + 0) * 2 + 0, _link_ea(2, 0), 4]
    assert out["path"].tolist() == path + path
    assert out["bw"].tolist() == [60, 60]
    # the pod's score is its rank in the original five-host ranking
    hosts = sorted(VIABLE)
    s = dict(zip(hosts, _score(method, rule, _rows(hosts))))
    assert out["pod_score"][1] == s[4]
    assert out["pod_score"][0] == 1.0  # pod 0 had a single viable host
    # the failed attempts left nothing behind: only host 4's path changed
    exp = res0.copy()
    for l in path:
        exp[l] -= 120
    assert np.array_equal(dc.state(O.LINK_RES), exp)
    assert dc.state(O.LINK_RES)[_link_ea(4, 0)] == 100


@pytest.mark.parametrize("method,rule", METHODS)
def test_every_candidate_fails_rejects_and_rolls_back(method, rule):
    """Pod 1 of 18 CPU: only hosts 8 and 9 are viable and both commits fail,
    so the request is rejected and pod 0's placement on host 0 is undone."""
    dc = _dc(method, rule)
    before = [dc.state(f) for f in (O.FREE_CPU, O.FREE_MEM, O.CTR, O.LINK_RES)]
    out = dc.schedule(_request(cpu_pod1=18))
    assert out["status"] == O.REJECTED
    assert out["n_decisions"] == 2
    assert np.all(out["host"] == -1) and np.all(out["bw"] == 0) and np.all(out["path"] == -1)
    after = [dc.state(f) for f in (O.FREE_CPU, O.FREE_MEM, O.CTR, O.LINK_RES)]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)

"""Pins of the oracle's discrete-event simulation with queueing: a
hand-worked queue, strict FCFS order of the starts, and capacities respected
at every step (reconstructed from the placements themselves)."""
import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W


def _one(cpu, mem=1):
    return {"cpu_min": np.array([cpu], np.int32), "cpu_max": np.array([cpu], np.int32),
            "mem_min": np.array([mem], np.int32), "mem_max": np.array([mem], np.int32),
            "pod": np.array([0], np.int32), "src": np.zeros(0, np.int32),
            "dst": np.zeros(0, np.int32), "bw_min": np.zeros(0, np.int32),
            "bw_max": np.zeros(0, np.int32)}


def test_hand_worked_queue():
    """Two 8-CPU hosts, five requests that each need a whole host, submitted
    at steps 0,0,0,1,1 with running times 3,2,5,1,1: r0, r1 start at 0; r2
    waits for r1 (leaves at 2); r3 for r0 (leaves at 3); r4 for r3 (leaves at
    4).  Blocked heads are retried only after a departure: r2, r3 and r4 take
    two attempts each."""
    dc = O.OracleDC(2, 8, 16, 1000, 4, O.TOPSIS, O.RATIO, [0.25] * 4, None, None, None)
    outs, start = dc.simulate([_one(8)] * 5, [0, 0, 0, 1, 1], [3, 2, 5, 1, 1], 20)
    assert list(start) == [0, 0, 2, 3, 4]
    assert [o["status"] for o in outs] == [O.ACCEPTED] * 5
    assert [o["n_decisions"] for o in outs] == [1, 1, 2, 2, 2]


def test_never_started_requests_are_rejected():
    dc = O.OracleDC(2, 8, 16, 1000, 4, O.TOPSIS, O.RATIO, [0.25] * 4, None, None, None)
    outs, start = dc.simulate([_one(8), _one(8), _one(8)], [0, 0, 0], [10, 10, 10], 5)
    assert list(start) == [0, 0, -1]
    assert outs[2]["status"] == O.REJECTED and np.all(outs[2]["host"] == -1)


@pytest.mark.parametrize("method", [O.TOPSIS, O.AHP, O.BF, O.WF])
def test_fcfs_order_and_capacity_every_step(method):
    """k=4 fat-tree of 8-CPU hosts under heavy load: starts follow the FCFS
    order (non-decreasing, never before submission, none after a request
    that never starts), and at every step the running requests' containers
    and path bandwidths fit the hosts and links."""
    T = 120
    wl, sub, dur = W.simulation(seed=9, k=4, n_requests=150, n_steps=T, max_duration=30,
                                host_cpu=8, host_mem=16, link_mbps=100, method=method)
    inst = wl.instances[0]
    reqs = [inst.reqs.request(r) for r in range(inst.reqs.n)]
    dc = O.OracleDC.from_instance(inst)
    outs, start = dc.simulate(reqs, sub, dur, T)
    order = np.lexsort((np.arange(len(sub)), sub))
    st = start[order]
    blocked = False
    prev = -1
    for i, r in enumerate(order):
        if st[i] < 0:
            blocked = True
            continue
        assert not blocked
        assert st[i] >= sub[r] and st[i] >= prev
        prev = st[i]
    H = inst.hosts
    for t in range(T):
        cpu = np.zeros(H, np.int64)
        mem = np.zeros(H, np.int64)
        link = np.zeros(3 * H, np.int64)
        for r, o in enumerate(outs):
            if start[r] < 0 or not (start[r] <= t < start[r] + dur[r]):
                continue
            np.add.at(cpu, o["host"], o["cpu"])
            np.add.at(mem, o["host"], o["mem"])
            for e in range(len(reqs[r]["src"])):
                for l in o["path"][6 * e:6 * e + 6]:
                    if l >= 0:
                        link[l] += o["bw"][e]
        assert np.all(cpu <= inst.host_cpu) and np.all(mem <= inst.host_mem)
        assert np.all(link <= inst.link_mbps)
    assert np.sum(start >= 0) < len(start)  # the load does queue and block

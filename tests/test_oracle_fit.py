"""Pins of the best-fit / worst-fit comparators of the oracle: best fit packs
(fills the tightest host first), worst fit spreads (takes the emptiest host),
both checked against a brute force over exact fractions of free capacity."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W


def _singletons(n, cpu=1, mem=1):
    return {
        "cpu_min": np.full(n, cpu, np.int32), "cpu_max": np.full(n, cpu, np.int32),
        "mem_min": np.full(n, mem, np.int32), "mem_max": np.full(n, mem, np.int32),
        "pod": np.arange(n, dtype=np.int32),
        "src": np.zeros(0, np.int32), "dst": np.zeros(0, np.int32),
        "bw_min": np.zeros(0, np.int32), "bw_max": np.zeros(0, np.int32),
    }


def _dc(method, k=4, cpu=8, mem=16, pre_cpu=None, pre_mem=None):
    return O.OracleDC(k, cpu, mem, 1000, 4, method, O.RATIO, [0.25] * 4, pre_cpu, pre_mem, None)


def test_best_fit_packs():
    """Empty k=4 fat-tree of 8-CPU hosts, 20 one-CPU containers one per pod:
    best fit fills host 0, then host 1, then host 2."""
    dc = _dc(O.BF)
    out = dc.schedule(_singletons(20))
    assert out["status"] == O.ACCEPTED
    assert list(out["host"]) == [0] * 8 + [1] * 8 + [2] * 4


def test_worst_fit_spreads():
    """Worst fit puts the first 16 containers on 16 distinct hosts in index
    order, then wraps around."""
    dc = _dc(O.WF)
    out = dc.schedule(_singletons(20))
    assert list(out["host"]) == list(range(16)) + [0, 1, 2, 3]


def _brute_choice(free_c, free_m, cap_c, cap_m, need_c, need_m, method):
    best, key = -1, None
    for u in range(len(free_c)):
        if free_c[u] < need_c or free_m[u] < need_m:
            continue
        s = Fraction(int(free_c[u]), cap_c) + Fraction(int(free_m[u]), cap_m)
        k = s if method == O.WF else -s
        if key is None or k > key:
            best, key = u, k
    return best


@pytest.mark.parametrize("method", [O.BF, O.WF])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fit_matches_brute_force(method, seed):
    """Random pre-load on k=4 (32 CPU / 64 memory hosts), singleton
    containers without links: every choice equals the brute-force extremum of
    free_cpu / 32 + free_mem / 64 (exact fractions, lowest index on ties),
    and the reported pod score is that host's (free_cpu/32 + free_mem/64)/2."""
    rng = np.random.default_rng(seed)
    H = 16
    pc = rng.integers(0, 30, H).astype(np.int32)
    pm = rng.integers(0, 60, H).astype(np.int32)
    dc = _dc(method, cpu=32, mem=64, pre_cpu=pc, pre_mem=pm)
    free_c, free_m = 32 - pc, 64 - pm
    for step in range(25):
        c, m = int(rng.integers(1, 5)), int(rng.integers(1, 9))
        q = _singletons(1, c, m)
        exp = _brute_choice(free_c, free_m, 32, 64, c, m, method)
        out = dc.schedule(q)
        if exp < 0:
            assert out["status"] == O.REJECTED
            continue
        assert out["host"][0] == exp
        assert out["pod_score"][0] == (free_c[exp] / 32 + free_m[exp] / 64) / 2
        free_c[exp] -= c
        free_m[exp] -= m


@pytest.mark.parametrize("method", [O.BF, O.WF])
def test_fit_placements_are_feasible(method):
    """Network requests on a pre-loaded k=8 fat-tree: every accepted
    placement respects capacities, and every link path carries at least its
    bw_min on links that never go negative (the commit is shared)."""
    inst = W.k16(seed=5, k=8, n_requests=30, method=method).instances[0]
    dc = O.OracleDC.from_instance(inst)
    for r in range(inst.reqs.n):
        dc.schedule(inst.reqs.request(r))
    assert np.all(dc.state(O.FREE_CPU) >= 0) and np.all(dc.state(O.FREE_MEM) >= 0)
    assert np.all(dc.state(O.LINK_RES) >= 0)

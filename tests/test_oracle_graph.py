"""Pins of the oracle's widest shortest paths on general graphs: brute force
over every simple path on small random graphs, and agreement with the
fat-tree path rule (lowest aggregation, then lowest core) of the scheduler
on fat-trees with random residuals."""
import itertools

import numpy as np
import pytest

import oracle as O


def _brute(V, lu, lv, res, s, t):
    """Every simple s -> t path by depth-first search; the fewest hops, then
    the largest bottleneck, then the smallest node sequence."""
    adj = {v: [] for v in range(V)}
    for l, (a, b) in enumerate(zip(lu, lv)):
        adj[a].append((b, l))
        adj[b].append((a, l))
    best = None

    def dfs(v, seen, nodes, links, bott):
        nonlocal best
        if v == t:
            key = (len(links), -bott, tuple(nodes))
            if best is None or key < best[0]:
                best = (key, list(nodes), list(links), bott)
            return
        if best is not None and len(links) >= best[0][0]:
            return
        for n, l in adj[v]:
            if n in seen:
                continue
            seen.add(n)
            nodes.append(n)
            links.append(l)
            dfs(n, seen, nodes, links, min(bott, int(res[l])))
            nodes.pop()
            links.pop()
            seen.discard(n)

    dfs(s, {s}, [s], [], 2 ** 31 - 1)
    return best


def _random_graph(rng, V, p):
    lu, lv = [], []
    for a, b in itertools.combinations(range(V), 2):
        if rng.random() < p:
            lu.append(a)
            lv.append(b)
    res = rng.integers(0, 6, len(lu))  # few distinct values: many ties
    return lu, lv, res


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_small_graphs(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(5, 10))
    lu, lv, res = _random_graph(rng, V, 0.4)
    g = O.OracleGraph(V, lu, lv, res)
    for s in range(V):
        for t in range(V):
            h, b, nodes, links = g.widest_path(s, t)
            if s == t:
                assert h == 0 and list(nodes) == [s]
                continue
            exp = _brute(V, lu, lv, res, s, t)
            if exp is None:
                assert h == -1
                continue
            assert h == len(exp[2]) and b == exp[3]
            assert list(nodes) == exp[1] and list(links) == exp[2]


@pytest.mark.parametrize("k", [4, 6])
def test_fattree_agrees_with_scheduler_rule(k):
    """On a fat-tree with random residuals the general search returns the
    path of the fat-tree rule (orc_widest_path), link for link."""
    rng = np.random.default_rng(k)
    H = k ** 3 // 4
    res = rng.integers(0, 50, 3 * H).astype(np.int32)
    V, lu, lv = O.fattree_graph(k, res)
    g = O.OracleGraph(V, lu, lv, res)
    dc = O.OracleDC(k, 32, 64, 100, 4, O.TOPSIS, O.RATIO, [0.25] * 4, None, None,
                    (100 - res).astype(np.int32))
    for _ in range(60):
        s, t = (int(x) for x in rng.choice(H, 2, replace=False))
        b_ft, links_ft = dc.widest_path(s, t)[:2]
        h, b, nodes, links = g.widest_path(s, t)
        assert b == b_ft
        assert list(links) == [l for l in links_ft if l >= 0]


def test_unreachable_and_validation():
    g = O.OracleGraph(4, [0, 2], [1, 3], [5, 5])
    assert g.widest_path(0, 3)[0] == -1
    with pytest.raises(ValueError):
        O.OracleGraph(3, [0, 1], [1, 0], [1, 1])  # duplicate link
    with pytest.raises(ValueError):
        O.OracleGraph(3, [0], [0], [1])  # loop

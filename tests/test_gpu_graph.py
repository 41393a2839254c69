"""Parity of the device widest-shortest-path search on general graphs with
the oracle: hops, bottleneck and the link sequence of every pair equal, on
random graphs (many ties), on fat-trees (where both follow the scheduler's
path rule) and for unreachable and trivial pairs.  Needs a GPU."""
import itertools

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    import torch

    torch.cuda.set_device(0)
    from paper_1909_07673_gb300 import dcsched

    dcsched.lib()
    return dcsched


def _compare(ds, V, lu, lv, res, pairs, max_hops=16):
    g = ds.Graph(V, lu, lv, res)
    og = O.OracleGraph(V, lu, lv, res)
    src = np.array([p[0] for p in pairs], np.int32)
    dst = np.array([p[1] for p in pairs], np.int32)
    hops, bott, links = g.widest_paths(src, dst, max_hops)
    for i, (s, t) in enumerate(pairs):
        h, b, nodes, ol = og.widest_path(int(s), int(t), max_nodes=max_hops + 1)
        assert hops[i] == h, (s, t)
        if h < 0:
            assert bott[i] == -1
            continue
        assert bott[i] == b, (s, t)
        assert list(links[i][:h]) == list(ol), (s, t)
        assert np.all(links[i][h:] == -1)
    g.close()


@pytest.mark.parametrize("seed", range(4))
def test_random_graphs_all_pairs(ds, seed):
    rng = np.random.default_rng(100 + seed)
    V = int(rng.integers(20, 60))
    lu, lv = [], []
    for a, b in itertools.combinations(range(V), 2):
        if rng.random() < 0.08:
            lu.append(a)
            lv.append(b)
    res = rng.integers(0, 5, len(lu))
    pairs = [(s, t) for s in range(V) for t in range(V)]
    _compare(ds, V, lu, lv, res, pairs)


@pytest.mark.parametrize("k", [4, 8, 16])
def test_fattree_graphs(ds, k):
    rng = np.random.default_rng(k)
    H = k ** 3 // 4
    res = rng.integers(0, 40, 3 * H).astype(np.int32)
    V, lu, lv = O.fattree_graph(k, res)
    pairs = [tuple(int(x) for x in rng.choice(H, 2, replace=False)) for _ in range(300)]
    pairs += [(0, 0), (H - 1, H - 1)]
    _compare(ds, V, lu, lv, res, pairs)


def test_set_residual_and_grid_loop(ds):
    """More pairs than resident blocks (the grid loops), then new residuals."""
    k = 8
    H = k ** 3 // 4
    rng = np.random.default_rng(7)
    res = rng.integers(0, 40, 3 * H).astype(np.int32)
    V, lu, lv = O.fattree_graph(k, res)
    g = ds.Graph(V, lu, lv, res)
    pairs = rng.integers(0, H, (2000, 2)).astype(np.int32)
    res2 = rng.integers(0, 40, 3 * H).astype(np.int32)
    g.set_residual(res2)
    hops, bott, links = g.widest_paths(pairs[:, 0], pairs[:, 1], 8)
    og = O.OracleGraph(V, lu, lv, res2)
    for i in range(0, 2000, 7):
        h, b, _, ol = og.widest_path(int(pairs[i, 0]), int(pairs[i, 1]))
        assert hops[i] == h and bott[i] == b
        assert list(links[i][:max(h, 0)]) == list(ol)
    g.close()


def test_graph_validation(ds):
    with pytest.raises(ds.DcError):
        ds.Graph(3, [0, 1], [1, 0], [1, 1])  # duplicate link
    with pytest.raises(ds.DcError):
        ds.Graph(3, [0], [3], [1])  # node out of range

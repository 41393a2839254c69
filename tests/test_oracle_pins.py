"""Pins of the FP64 oracle against what the paper and the mathematics fix:
topology counts of Sec. IV-B.1, brute-force widest shortest paths, the
hand-worked TOPSIS and AHP examples under tests/golden/, closed forms,
special cases and invariants.  CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1909_07673_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


# ---------------------------------------------------------------- topology

def test_fattree_counts_golden():
    for k, hosts, switches, links in _rows("fattree_counts.txt"):
        d = O.fattree_dims(int(k))
        assert d["hosts"] == int(hosts)
        assert d["edge"] + d["agg"] + d["core"] == int(switches)
        assert d["links"] == int(links)


@pytest.mark.parametrize("k", [2, 4, 6, 8, 16, 48])
def test_fattree_counts_formula(k):
    d = O.fattree_dims(k)
    assert d["hosts"] == k ** 3 // 4
    assert d["edge"] + d["agg"] + d["core"] == 5 * k * k // 4
    assert d["links"] == 3 * k ** 3 // 4


@pytest.mark.parametrize("k", [4, 6, 8])
def test_graph_structure_matches_numbering(k):
    """Every link id of the documented numbering is used exactly once by the
    independently built graph, and degrees are those of a k-port fat-tree."""
    pytest.importorskip("networkx")
    from fattree_ref import build

    G, lid = build(k)
    assert sorted(lid.values()) == list(range(3 * k ** 3 // 4))
    for n, deg in G.degree():
        assert deg == (1 if n[0] == "h" else k if n[0] in "ea" else k)


@pytest.mark.parametrize("k,levels", [(4, 3), (4, 60), (6, 5), (8, 4)])
def test_widest_shortest_path_bruteforce(k, levels):
    """Bottleneck, hop count, chosen links and the (a, c) tie break against
    enumeration of all shortest paths of the networkx graph.  Few residual
    levels force many ties."""
    pytest.importorskip("networkx")
    from fattree_ref import build, widest_shortest

    G, lid = build(k)
    H = k ** 3 // 4
    rng = np.random.default_rng(100 + k + levels)
    cap = 1000
    res = rng.integers(0, levels, 3 * H) * (cap // levels)
    dc = O.OracleDC(k, 8, 8, cap, 4, O.TOPSIS, O.RATIO, (0.25,) * 4,
                    pre_link=(cap - res).astype(np.int32))
    assert np.array_equal(dc.state(O.LINK_RES), res)
    pairs = [(u, v) for u in range(H) for v in range(H) if u != v]
    idx = rng.choice(len(pairs), size=min(len(pairs), 150), replace=False)
    for i in idx:
        u, v = pairs[i]
        b, links, hops = dc.widest_path(u, v)
        bb, bl, bh = widest_shortest(G, lid, res, u, v)
        assert (b, hops) == (bb, bh), (u, v)
        assert list(links[:hops]) == bl, (u, v)
        assert all(x == -1 for x in links[hops:])


# ---------------------------------------------------------------- TOPSIS

def test_topsis_hand_example():
    x = [[3, 0], [4, 1], [0, 1]]
    cl = O.topsis(x, [0.5, 0.5])
    exp = {}
    for host, expr in _rows("topsis_3x2.txt"):
        exp[int(host)] = eval(expr, {"sqrt": math.sqrt})
    for h, v in exp.items():
        assert cl[h] == pytest.approx(v, rel=1e-14, abs=1e-15)


def test_topsis_range_and_dominance():
    rng = np.random.default_rng(1)
    for _ in range(50):
        F, C = int(rng.integers(2, 40)), int(rng.choice([4, 6]))
        x = rng.integers(0, 50, (F, C))
        w = rng.random(C) + 0.01
        cl = O.topsis(x, w)
        assert np.all(cl >= 0) and np.all(cl <= 1)
        # a host at or above every column maximum is the ideal: closeness 1
        x2 = np.vstack([x, x.max(axis=0)])
        assert O.topsis(x2, w)[-1] == 1.0
        # a host at every column minimum is the anti-ideal: closeness 0
        x3 = np.vstack([x, x.min(axis=0)])
        if np.any(x.max(axis=0) != x.min(axis=0)):
            assert O.topsis(x3, w)[-1] == 0.0


def test_topsis_scale_and_permutation_invariance():
    rng = np.random.default_rng(2)
    x = rng.integers(1, 100, (25, 6))
    w = np.array([0.1, 0.2, 0.3, 0.1, 0.2, 0.1])
    cl = O.topsis(x, w)
    xs = x * np.array([1, 3, 7, 2, 5, 11])  # positive per-criterion scaling
    assert np.allclose(O.topsis(xs, w), cl, rtol=1e-12, atol=1e-14)
    perm = rng.permutation(len(x))
    assert np.array_equal(O.topsis(x[perm], w), cl[perm])


def test_topsis_degenerate_cases():
    assert O.topsis([[5, 5]], [0.5, 0.5])[0] == 1.0          # single viable host
    assert np.all(O.topsis([[2, 3]] * 4, [0.5, 0.5]) == 1.0)  # identical hosts
    cl = O.topsis([[0, 1], [0, 2]], [0.5, 0.5])              # an all-zero column
    assert cl[1] == 1.0 and cl[0] == 0.0
    # weight 0 removes a criterion
    a = O.topsis([[1, 9], [2, 1]], [1.0, 0.0])
    assert a[1] == 1.0 and a[0] == 0.0


def test_topsis_one_criterion_closed_form():
    """With one criterion the closeness is (x - min) / (max - min)."""
    x = np.array([[3], [7], [5], [11], [3]])
    cl = O.topsis(x, [1.0])
    exp = (x[:, 0] - 3) / 8.0
    assert np.allclose(cl, exp, rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------- AHP

def test_ahp_hand_example():
    vals = {}
    for rule, *ps in _rows("ahp_3.txt"):
        vals[rule] = [float(Fraction(p)) for p in ps]
    x = [[0], [1], [3]]
    assert np.allclose(O.ahp(x, [1.0], O.DIFF), vals["diff"], rtol=1e-14)
    assert np.allclose(O.ahp_literal(x, [1.0], O.DIFF), vals["diff"], rtol=1e-14)
    assert np.allclose(O.ahp(x, [1.0], O.RATIO), vals["ratio"], rtol=1e-15)
    assert np.allclose(O.ahp_literal(x, [1.0], O.RATIO), vals["ratio"], rtol=1e-14)


def test_ahp_ratio_closed_form_vs_literal_matrix():
    """A ratio-scale (consistent) AHP priority equals x_i / sum(x)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        F, C = int(rng.integers(1, 30)), int(rng.choice([4, 6]))
        x = rng.integers(0, 40, (F, C))
        w = rng.random(C) + 0.05
        pg = O.ahp(x, w, O.RATIO)
        assert np.allclose(O.ahp_literal(x, w, O.RATIO), pg, rtol=1e-12)
        L1 = w / w.sum()
        exp = ((x + 1) / (x + 1).sum(axis=0) * L1).sum(axis=1)
        assert np.allclose(pg, exp, rtol=1e-13)
        assert pg.sum() == pytest.approx(1.0, rel=1e-12)


def test_ahp_weights():
    w = np.array([0.17, 0.17, 0.5, 0.16])
    assert np.allclose(O.ahp_weights(w, O.RATIO), w / w.sum(), rtol=1e-15)
    # DIFF on the weights: literal rule, rows of a column-normalised
    # reciprocal matrix average to a probability vector
    l1 = O.ahp_weights(w, O.DIFF)
    assert l1.sum() == pytest.approx(1.0, rel=1e-14)
    assert l1[0] == l1[1]  # equal weights compare as equals
    # equal weights give equal priorities under both rules
    assert np.allclose(O.ahp_weights([0.25] * 4, O.DIFF), 0.25, rtol=1e-15)


def test_ahp_diff_grouped_fixed_point_vs_literal():
    rng = np.random.default_rng(4)
    for _ in range(30):
        F, C = int(rng.integers(1, 60)), int(rng.choice([4, 6]))
        hi = int(rng.choice([2, 5, 40, 3000]))
        x = rng.integers(0, hi, (F, C))
        w = rng.random(C) + 0.05
        a = O.ahp(x, w, O.DIFF)
        b = O.ahp_literal(x, w, O.DIFF)
        assert np.allclose(a, b, rtol=1e-12, atol=0), (F, hi)
        assert a.sum() == pytest.approx(1.0, rel=1e-12)


def test_ahp_diff_all_equal_is_uniform():
    for F in (1, 2, 7, 64):
        x = np.full((F, 4), 9)
        assert np.allclose(O.ahp(x, [0.25] * 4, O.DIFF), 1.0 / F, rtol=1e-15)


def test_ahp_diff_translation_invariance():
    """The difference reading (Sec. V-B) compares hosts by x_i - x_j only, so
    adding a constant to a criterion's column changes no priority (exactly:
    the differences are integers).  The ratio reading does not have this
    property, nor would a difference rule with an offset on one side."""
    rng = np.random.default_rng(6)
    for _ in range(20):
        F, C = int(rng.integers(2, 30)), int(rng.choice([4, 6]))
        x = rng.integers(0, 60, (F, C))
        w = rng.random(C) + 0.05
        shift = rng.integers(0, 500, C)
        assert np.array_equal(O.ahp(x + shift, w, O.DIFF), O.ahp(x, w, O.DIFF))
    x = np.array([[0, 3], [1, 1], [4, 2]])
    assert not np.allclose(O.ahp(x + 7, [0.5, 0.5], O.RATIO), O.ahp(x, [0.5, 0.5], O.RATIO))


def test_ahp_diff_dominance():
    """Under the difference reading a_ij grows with x_i - x_j, so a host at
    least as good as another in every criterion (all benefit criteria) has at
    least its priority, and strictly more when it is better in a criterion
    of positive weight and some third host separates them.  A reversed
    reciprocal (a_ij = 1 / d for d > 0) breaks this."""
    rng = np.random.default_rng(8)
    for _ in range(200):
        F, C = int(rng.integers(2, 20)), int(rng.choice([4, 6]))
        x = rng.integers(0, 25, (F, C))
        w = rng.random(C) + 0.05
        x[0] = np.maximum(x[0], x[1])
        p = O.ahp(x, w, O.DIFF)
        assert p[0] >= p[1]
    # hand case: host 0 better than host 1 in the first criterion only
    x = np.array([[5, 2], [3, 2], [0, 0]])
    p = O.ahp(x, [0.5, 0.5], O.DIFF)
    assert p[0] > p[1] > p[2]


def test_ahp_permutation_invariance():
    rng = np.random.default_rng(5)
    x = rng.integers(0, 500, (40, 6))
    w = rng.random(6) + 0.1
    perm = rng.permutation(40)
    for rule in (O.RATIO, O.DIFF):
        assert np.array_equal(O.ahp(x[perm], w, rule), O.ahp(x, w, rule)[perm])


def test_table4_weights():
    rows = {r[0]: tuple(float(v) for v in r[1:]) for r in _rows("weights_table4.txt")}
    for name, ws in rows.items():
        assert W.WEIGHTS[4][name] == ws
        assert sum(ws) == pytest.approx(1.0, abs=1e-12)
    for ws in W.WEIGHTS[6].values():
        assert sum(ws) == pytest.approx(1.0, abs=1e-12)

"""Independent fat-tree graph for the tests (networkx), built from the
structural description of Sec. IV-B.1 and the cited three-tier fat-tree:
k pods, each with k/2 edge and k/2 aggregation switches fully meshed; each
edge switch serves k/2 hosts; (k/2)^2 core switches, core (a, c) linked to
aggregation switch a of every pod.

Link ids follow the documented numbering of the scheduler's API (one
undirected residual per link): host links first (id = host index), then
edge-aggregation links, then aggregation-core links.
"""
import itertools


def build(k):
    import networkx as nx

    h2 = k // 2
    H = k ** 3 // 4
    G = nx.Graph()
    lid = {}
    host = 0
    for p in range(k):
        for j in range(h2):
            e = ("e", p, j)
            for _ in range(h2):
                G.add_edge(("h", host), e)
                lid[frozenset((("h", host), e))] = host
                host += 1
    for p in range(k):
        for j in range(h2):
            eg = p * h2 + j
            for a in range(h2):
                n1, n2 = ("e", p, j), ("a", p, a)
                G.add_edge(n1, n2)
                lid[frozenset((n1, n2))] = H + eg * h2 + a
    for p in range(k):
        for a in range(h2):
            for c in range(h2):
                n1, n2 = ("a", p, a), ("c", a, c)
                G.add_edge(n1, n2)
                lid[frozenset((n1, n2))] = 2 * H + (p * h2 + a) * h2 + c
    return G, lid


def path_links(lid, path):
    return [lid[frozenset((path[i], path[i + 1]))] for i in range(len(path) - 1)]


def path_key(path):
    """(a, c) of a path: the aggregation index and the core index it uses."""
    a = c = -1
    for n in path:
        if n[0] == "a":
            a = n[2]
        if n[0] == "c":
            c = n[2]
    return (a, c)


def widest_shortest(G, lid, res, u, v):
    """Brute force over all shortest paths: (bottleneck, links, hops) of the
    path with the largest bottleneck, ties to the lowest (a, c)."""
    import networkx as nx

    best = None
    for p in nx.all_shortest_paths(G, ("h", u), ("h", v)):
        links = path_links(lid, p)
        b = min(int(res[x]) for x in links)
        key = (-b, path_key(p))
        if best is None or key < best[0]:
            best = (key, b, links, len(p) - 1)
    return best[1], best[2], best[3]


def all_shortest_link_sets(G, lid, u, v):
    import networkx as nx

    return [path_links(lid, p) for p in nx.all_shortest_paths(G, ("h", u), ("h", v))]

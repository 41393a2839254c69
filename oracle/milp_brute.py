"""Exhaustive checks of placements against the MILP of Sec. III.

TEST INFRASTRUCTURE ONLY.  Written independently of oracle.c: it knows the
fat-tree only through a networkx graph supplied by the caller (nodes
("h", i) for hosts, a dict mapping each undirected link to its id) and checks
the constraints of Eqs. 4-8, the single-host constraint and the path
(flow-conservation) constraint of Sec. III-B on a given placement.  For tiny
instances it also enumerates every pod-to-host map and every shortest-path
choice, to report whether any feasible placement exists and the best value of
the objective of Eq. 3 among the enumerated ones.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Sequence

import numpy as np


def check_placement(G, lid: Dict, free_cpu, free_mem, res, req: Dict[str, np.ndarray],
                    out: Dict[str, np.ndarray]) -> List[str]:
    """Returns the list of violated constraints (empty when feasible)."""
    import networkx as nx

    bad: List[str] = []
    n = len(req["pod"])
    H = len(free_cpu)
    host = out["host"]
    use_cpu = np.zeros(H, np.int64)
    use_mem = np.zeros(H, np.int64)
    for i in range(n):
        u = int(host[i])
        if not 0 <= u < H:
            bad.append("container %d not on a single host" % i)
            continue
        if not req["cpu_min"][i] <= out["cpu"][i] <= req["cpu_max"][i]:
            bad.append("Eq.6 cpu of container %d" % i)
        if not req["mem_min"][i] <= out["mem"][i] <= req["mem_max"][i]:
            bad.append("Eq.6 mem of container %d" % i)
        use_cpu[u] += out["cpu"][i]
        use_mem[u] += out["mem"][i]
    for i in range(n):
        for j in range(n):
            if req["pod"][i] == req["pod"][j] and host[i] != host[j]:
                bad.append("Eq.8 pod integrity %d/%d" % (i, j))
    if np.any(use_cpu > np.asarray(free_cpu)) or np.any(use_mem > np.asarray(free_mem)):
        bad.append("Eq.4 host capacity")
    use_link = np.zeros(len(res), np.int64)
    id2edge = {v: tuple(k) for k, v in lid.items()}
    for e in range(len(req["src"])):
        hs, ht = int(host[req["src"][e]]), int(host[req["dst"][e]])
        links = [int(x) for x in out["path"][6 * e:6 * e + 6] if x >= 0]
        bw = int(out["bw"][e])
        if not req["bw_min"][e] <= bw <= req["bw_max"][e]:
            bad.append("Eq.7 bandwidth of link %d" % e)
        if hs == ht:
            if links:
                bad.append("link %d between co-located containers uses the network" % e)
            continue
        # path constraint: the links form a walk from host(src) to host(dst)
        cur = ("h", hs)
        ok = True
        for x in links:
            a, b = id2edge[x]
            if cur == a:
                cur = b
            elif cur == b:
                cur = a
            else:
                ok = False
                break
        if not ok or cur != ("h", ht):
            bad.append("path of link %d is not a path between its hosts" % e)
        elif len(links) != nx.shortest_path_length(G, ("h", hs), ("h", ht)):
            bad.append("path of link %d is not a shortest path" % e)
        for x in links:
            use_link[x] += bw
    if np.any(use_link > np.asarray(res)):
        bad.append("Eq.5 link capacity")
    return bad


def objective(alpha: float, req, out, n_hosts_active: int, H: int, n_links_active: int,
              L: int) -> float:
    """Eq. 3 for one request: alpha * utility loss + (1 - alpha) * fragmentation."""
    n = len(req["pod"])
    u_i = sum((out["cpu"][i] / req["cpu_max"][i] + out["mem"][i] / req["mem_max"][i]) / 2
              for i in range(n) if req["cpu_max"][i] > 0 and req["mem_max"][i] > 0)
    u_ij = sum(out["bw"][e] / req["bw_max"][e] for e in range(len(req["src"]))
               if req["bw_max"][e] > 0)
    return alpha * ((n - u_i) + (len(req["src"]) - u_ij)) + (1 - alpha) * (
        n_hosts_active / H + n_links_active / L)


def exhaustive_feasible(G, lid, free_cpu, free_mem, res, req, max_maps: int = 200000
                        ) -> Optional[bool]:
    """True when some pod-to-host map with minimum allocations and some choice
    of shortest paths satisfies Eqs. 4-8; None when the search is too large."""
    import networkx as nx

    H = len(free_cpu)
    pods = sorted(set(int(p) for p in req["pod"]))
    if H ** len(pods) > max_maps:
        return None
    members = {g: [i for i in range(len(req["pod"])) if req["pod"][i] == g] for g in pods}
    paths: Dict = {}

    def shortest(hs, ht):
        if (hs, ht) not in paths:
            paths[(hs, ht)] = [[lid[frozenset((p[i], p[i + 1]))] for i in range(len(p) - 1)]
                               for p in nx.all_shortest_paths(G, ("h", hs), ("h", ht))]
        return paths[(hs, ht)]

    res = [int(x) for x in res]
    for hosts in itertools.product(range(H), repeat=len(pods)):
        cpu = [0] * H
        mem = [0] * H
        for g, u in zip(pods, hosts):
            for i in members[g]:
                cpu[u] += int(req["cpu_min"][i])
                mem[u] += int(req["mem_min"][i])
        if any(cpu[u] > free_cpu[u] or mem[u] > free_mem[u] for u in set(hosts)):
            continue
        hmap = {g: u for g, u in zip(pods, hosts)}
        choices = []
        for e in range(len(req["src"])):
            hs, ht = hmap[int(req["pod"][req["src"][e]])], hmap[int(req["pod"][req["dst"][e]])]
            choices.append([[]] if hs == ht else shortest(hs, ht))
        for combo in itertools.product(*choices):
            use: Dict[int, int] = {}
            for e, links in enumerate(combo):
                for x in links:
                    use[x] = use.get(x, 0) + int(req["bw_min"][e])
            if all(v <= res[x] for x, v in use.items()):
                return True
    return False

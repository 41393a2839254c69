"""Seeded synthetic workloads for the scheduler.

This module only draws random inputs: data-center sizes, pre-load, tenant
requests (containers with [min, max] CPU and memory, pods, links with
[min, max] bandwidth) and, for the serving workload, arrival times and
departures.  It holds none of the scheduling arithmetic; both the CUDA path
and the FP64 oracle consume the arrays it returns.

The shapes follow the paper's synthetic workloads (Sec. IV-B and VI-A:
fat-tree data centers, homogeneous hosts, uniform container sizes, pods of a
few containers, link bandwidth requirements) scaled to the five benchmark
configurations:

  small    k=4 fat-tree, 10 requests of 2-8 containers, 4 criteria
  k16      k=16, 0-70 % pre-load, 1,000 requests of 4-64 containers, 6 criteria
  k48      k=48, 0-100 % pre-load, 200 requests of 64-512 containers in pods
           of 1-8, Pareto(1.5) inter-pod bandwidth, 6 criteria
  serving  64 k=16 instances, Poisson arrivals at 50k/s for 1 s, Zipf(1.1)
           over instances, 2-128 containers, exponential lifetimes
  batched  256 instances with k cycling over {8, 16, 24, 32}, 100 requests of
           4-256 containers each

Random numbers come from numpy's PCG64 generator seeded per workload; the
same seed gives the same arrays for a given numpy version.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

TOPSIS, AHP, BF, WF = 0, 1, 2, 3
RATIO, DIFF = 0, 1

# Table IV weighting schemes for the four criteria (CPU, RAM, fragmentation,
# bandwidth).  For six criteria (plus path bandwidth and locality) the same
# rule is kept: Flat shares equally, Clustering gives fragmentation 1/2,
# Network gives the two bandwidth criteria 1/2 together.
WEIGHTS: Dict[int, Dict[str, Tuple[float, ...]]] = {
    4: {
        "flat": (0.25, 0.25, 0.25, 0.25),
        "clustering": (0.17, 0.17, 0.5, 0.16),
        "network": (0.17, 0.17, 0.16, 0.5),
    },
    6: {
        "flat": (1 / 6,) * 6,
        "clustering": (0.1, 0.1, 0.5, 0.1, 0.1, 0.1),
        "network": (0.125, 0.125, 0.125, 0.25, 0.25, 0.125),
    },
}


def fattree_hosts(k: int) -> int:
    return k * k * k // 4


@dataclasses.dataclass
class RequestBatch:
    """Requests packed back to back: request r owns containers
    c_off[r]:c_off[r+1] and links e_off[r]:e_off[r+1] (container indices in
    src/dst are local to the request)."""

    c_off: np.ndarray
    e_off: np.ndarray
    cpu_min: np.ndarray
    cpu_max: np.ndarray
    mem_min: np.ndarray
    mem_max: np.ndarray
    pod: np.ndarray
    src: np.ndarray
    dst: np.ndarray
    bw_min: np.ndarray
    bw_max: np.ndarray

    @property
    def n(self) -> int:
        return len(self.c_off) - 1

    def request(self, r: int) -> Dict[str, np.ndarray]:
        c0, c1 = int(self.c_off[r]), int(self.c_off[r + 1])
        e0, e1 = int(self.e_off[r]), int(self.e_off[r + 1])
        return {
            "cpu_min": self.cpu_min[c0:c1], "cpu_max": self.cpu_max[c0:c1],
            "mem_min": self.mem_min[c0:c1], "mem_max": self.mem_max[c0:c1],
            "pod": self.pod[c0:c1],
            "src": self.src[e0:e1], "dst": self.dst[e0:e1],
            "bw_min": self.bw_min[e0:e1], "bw_max": self.bw_max[e0:e1],
        }

    def n_pods(self, r: int) -> int:
        c0, c1 = int(self.c_off[r]), int(self.c_off[r + 1])
        return int(self.pod[c0:c1].max()) + 1 if c1 > c0 else 0

    def subset(self, rs: Sequence[int]) -> "RequestBatch":
        return pack_requests([self.request(int(r)) for r in rs])


def pack_requests(reqs: Sequence[Dict[str, np.ndarray]]) -> RequestBatch:
    c_off = np.zeros(len(reqs) + 1, np.int64)
    e_off = np.zeros(len(reqs) + 1, np.int64)
    for i, q in enumerate(reqs):
        c_off[i + 1] = c_off[i] + len(q["pod"])
        e_off[i + 1] = e_off[i] + len(q["src"])

    def cat(name):
        parts = [np.asarray(q[name], np.int32) for q in reqs]
        return np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(0, np.int32),
                                    dtype=np.int32)

    return RequestBatch(c_off, e_off, *(cat(n) for n in (
        "cpu_min", "cpu_max", "mem_min", "mem_max", "pod", "src", "dst", "bw_min", "bw_max")))


@dataclasses.dataclass
class Instance:
    """One data center and the FCFS stream of requests submitted to it."""

    k: int
    host_cpu: int
    host_mem: int
    link_mbps: int
    n_criteria: int
    method: int
    pair_rule: int
    weights: Tuple[float, ...]
    pre_cpu: Optional[np.ndarray]
    pre_mem: Optional[np.ndarray]
    pre_link: Optional[np.ndarray]
    reqs: RequestBatch
    # Optional interleaved stream of operations: (kind, request index) with
    # kind 0 = schedule, 1 = release.  None means "schedule every request".
    ops: Optional[List[Tuple[int, int]]] = None

    @property
    def hosts(self) -> int:
        return fattree_hosts(self.k)

    def config_dict(self) -> dict:
        return dict(k=self.k, host_cpu=self.host_cpu, host_mem=self.host_mem,
                    link_mbps=self.link_mbps, n_criteria=self.n_criteria,
                    method=self.method, pair_rule=self.pair_rule,
                    weights=tuple(self.weights))

    def with_method(self, method: int, pair_rule: int = RATIO,
                    weights: Optional[Sequence[float]] = None) -> "Instance":
        w = tuple(weights) if weights is not None else self.weights
        return dataclasses.replace(self, method=method, pair_rule=pair_rule, weights=w)


@dataclasses.dataclass
class Workload:
    name: str
    instances: List[Instance]
    # serving only: per request (global order) arrival time [s] and instance id
    arrival_s: Optional[np.ndarray] = None
    arrival_inst: Optional[np.ndarray] = None
    arrival_local: Optional[np.ndarray] = None  # request index inside its instance


# --------------------------------------------------------------------------
# primitive draws

def _connect(rng: np.random.Generator, n: int, ei: np.ndarray, ej: np.ndarray
             ) -> Tuple[np.ndarray, np.ndarray]:
    """Makes the graph on n nodes connected: for each node i in increasing
    order that is not yet connected to node 0, add a link (i, j) with j drawn
    uniformly from 0..i-1."""
    if n <= 1:
        return ei, ej
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in zip(ei.tolist(), ej.tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    add_i, add_j = [], []
    for i in range(1, n):
        if find(i) != find(0):
            j = int(rng.integers(0, i))
            add_i.append(i)
            add_j.append(j)
            parent[find(i)] = find(0)
    if add_i:
        ei = np.concatenate([ei, np.asarray(add_i, np.int64)])
        ej = np.concatenate([ej, np.asarray(add_j, np.int64)])
    return ei, ej


def _er_graph(rng: np.random.Generator, n: int, p: float) -> Tuple[np.ndarray, np.ndarray]:
    if n < 2:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    return _connect(rng, n, iu[keep].astype(np.int64), ju[keep].astype(np.int64))


def _bw_uniform(lo: int, hi: int):
    return lambda rng, m: rng.integers(lo, hi + 1, m)


def _bw_loguniform(hi: float):
    return lambda rng, m: np.maximum(1, np.floor(np.exp(rng.random(m) * math.log(hi)))).astype(np.int64)


def _bw_pareto(alpha: float, xm: float, cap: int):
    def draw(rng, m):
        u = 1.0 - rng.random(m)  # (0, 1]
        return np.minimum(cap, np.floor(xm / u ** (1.0 / alpha))).astype(np.int64)
    return draw


def gen_request(rng: np.random.Generator, n: int, *, p_edge: float, bw, max_pod: int = 1,
                cpu_hi: int = 4, mem_hi: int = 8, intervals: bool = False,
                intra_pod_links: bool = False) -> Dict[str, np.ndarray]:
    """n containers; CPU U{1..cpu_hi}, memory U{1..mem_hi}.  max_pod == 1 gives
    singleton pods and an Erdos-Renyi graph over containers; otherwise the
    containers are cut into consecutive pods of U{1..max_pod} and the
    Erdos-Renyi graph is drawn over pods, each pod pair joined by a link
    between random members.  Both graphs are made connected.  With
    intervals=True the minimum is drawn at or below the maximum (otherwise
    min = max)."""
    cpu_max = rng.integers(1, cpu_hi + 1, n)
    mem_max = rng.integers(1, mem_hi + 1, n)
    if intervals:
        cpu_min = np.maximum(0, cpu_max - rng.integers(0, 3, n))
        mem_min = np.maximum(0, mem_max - rng.integers(0, 5, n))
    else:
        cpu_min, mem_min = cpu_max.copy(), mem_max.copy()
    if max_pod <= 1:
        pod = np.arange(n)
        gi, gj = _er_graph(rng, n, p_edge)
        src, dst = gi, gj
    else:
        sizes = []
        tot = 0
        while tot < n:
            s = int(rng.integers(1, max_pod + 1))
            s = min(s, n - tot)
            sizes.append(s)
            tot += s
        P = len(sizes)
        starts = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        pod = np.repeat(np.arange(P), sizes)
        gi, gj = _er_graph(rng, P, p_edge)
        sz = np.asarray(sizes, np.int64)
        src = starts[gi] + (rng.random(len(gi)) * sz[gi]).astype(np.int64)
        dst = starts[gj] + (rng.random(len(gj)) * sz[gj]).astype(np.int64)
        if intra_pod_links:
            multi = np.nonzero(sz >= 2)[0]
            pick = multi[rng.random(len(multi)) < 0.5]
            src = np.concatenate([src, starts[pick]])
            dst = np.concatenate([dst, starts[pick] + 1])
    m = len(src)
    flip = rng.random(m) < 0.5
    s2 = np.where(flip, dst, src)
    d2 = np.where(flip, src, dst)
    bw_max = bw(rng, m).astype(np.int64)
    bw_min = np.maximum(0, bw_max - (rng.integers(0, bw_max // 2 + 1) if intervals else 0))
    return {
        "cpu_min": cpu_min.astype(np.int32), "cpu_max": cpu_max.astype(np.int32),
        "mem_min": mem_min.astype(np.int32), "mem_max": mem_max.astype(np.int32),
        "pod": pod.astype(np.int32),
        "src": s2.astype(np.int32), "dst": d2.astype(np.int32),
        "bw_min": np.asarray(bw_min, np.int32), "bw_max": bw_max.astype(np.int32),
    }


def gen_preload(rng: np.random.Generator, k: int, host_cpu: int, host_mem: int,
                link_mbps: int, util_hi: float):
    """Per-host and per-link used amounts floor(U[0, util_hi) * capacity),
    drawn independently for CPU, memory and every link."""
    H = fattree_hosts(k)
    pre_cpu = np.floor(rng.random(H) * util_hi * host_cpu).astype(np.int32)
    pre_mem = np.floor(rng.random(H) * util_hi * host_mem).astype(np.int32)
    pre_link = np.floor(rng.random(3 * H) * util_hi * link_mbps).astype(np.int32)
    return pre_cpu, pre_mem, pre_link


# --------------------------------------------------------------------------
# the five configurations

def small(seed: int = 0, method: int = TOPSIS, pair_rule: int = RATIO,
          scheme: str = "flat", n_requests: int = 10, intervals: bool = False) -> Workload:
    """k=4 (16 hosts, 1 Gbps), 32 CPU / 64 GB hosts, no pre-load, 10 requests
    of U{2..8} containers, singleton pods, Erdos-Renyi p=0.4 made connected,
    bandwidth U{10..200} Mbps, 4 criteria."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = [gen_request(rng, int(rng.integers(2, 9)), p_edge=0.4, bw=_bw_uniform(10, 200),
                        intervals=intervals) for _ in range(n_requests)]
    inst = Instance(4, 32, 64, 1000, 4, method, pair_rule, WEIGHTS[4][scheme],
                    None, None, None, pack_requests(reqs))
    return Workload("small", [inst])


def k16(seed: int = 1, method: int = TOPSIS, pair_rule: int = RATIO, scheme: str = "flat",
        n_requests: int = 1000, k: int = 16, intervals: bool = False,
        preload: float = 0.7) -> Workload:
    """k=16 (1,024 hosts, 10 Gbps), pre-load U[0, preload) per host resource
    and link (0.7 by default; 0: an empty data center, the same requests),
    n_requests of U{4..64} containers, singleton pods, Erdos-Renyi p=0.1 made
    connected, log-uniform 1-1000 Mbps, 6 criteria."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pre = gen_preload(rng, k, 32, 64, 10000, preload)
    reqs = [gen_request(rng, int(rng.integers(4, 65)), p_edge=0.1, bw=_bw_loguniform(1000.0),
                        intervals=intervals) for _ in range(n_requests)]
    inst = Instance(k, 32, 64, 10000, 6, method, pair_rule, WEIGHTS[6][scheme],
                    *pre, pack_requests(reqs))
    return Workload("k16", [inst])


def k48(seed: int = 2, method: int = TOPSIS, pair_rule: int = RATIO, scheme: str = "flat",
        n_requests: int = 200, k: int = 48) -> Workload:
    """k=48 (27,648 hosts, 40 Gbps), pre-load U[0, 1) per host resource and
    link (mean 50 %), n_requests of U{64..512} containers in pods of
    U{1..8}, Erdos-Renyi p=0.1 over pods made connected, Pareto(1.5, 10)
    bandwidth capped at 10,000 Mbps, 6 criteria."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pre = gen_preload(rng, k, 32, 64, 40000, 1.0)
    reqs = [gen_request(rng, int(rng.integers(64, 513)), p_edge=0.1, bw=_bw_pareto(1.5, 10.0, 10000),
                        max_pod=8, intra_pod_links=True) for _ in range(n_requests)]
    inst = Instance(k, 32, 64, 40000, 6, method, pair_rule, WEIGHTS[6][scheme],
                    *pre, pack_requests(reqs))
    return Workload("k48", [inst])


def batched(seed: int = 4, method: int = TOPSIS, pair_rule: int = RATIO, scheme: str = "flat",
            n_instances: int = 256, n_requests: int = 100, ks: Sequence[int] = (8, 16, 24, 32),
            size_hi: int = 256) -> Workload:
    """n_instances data centers, instance i a fat-tree with k = ks[i % len(ks)]
    (10 Gbps, pre-load U[0, 0.7) as in k16), each receiving n_requests of
    U{4..size_hi} containers (singleton pods, Erdos-Renyi p=0.1 made
    connected, log-uniform 1-1000 Mbps), 6 criteria."""
    rng = np.random.Generator(np.random.PCG64(seed))
    insts = []
    for i in range(n_instances):
        k = int(ks[i % len(ks)])
        pre = gen_preload(rng, k, 32, 64, 10000, 0.7)
        reqs = [gen_request(rng, int(rng.integers(4, size_hi + 1)), p_edge=0.1,
                            bw=_bw_loguniform(1000.0)) for _ in range(n_requests)]
        insts.append(Instance(k, 32, 64, 10000, 6, method, pair_rule, WEIGHTS[6][scheme],
                              *pre, pack_requests(reqs)))
    return Workload("batched", insts)


def serving(seed: int = 3, method: int = TOPSIS, pair_rule: int = RATIO, scheme: str = "flat",
            n_instances: int = 64, rate_per_s: float = 50000.0, duration_s: float = 1.0,
            k: int = 16, size_lo: int = 2, size_hi: int = 128, zipf_s: float = 1.1,
            mean_life: float = 100.0) -> Workload:
    """n_instances k=16 data centers (pre-load as k16).  Requests arrive as a
    Poisson process at rate_per_s for duration_s; each goes to instance
    Zipf(zipf_s) over the instances, has U{size_lo..size_hi} containers
    (singleton pods, Erdos-Renyi p=0.1 made connected, log-uniform
    1-1000 Mbps) and departs after Exp(mean_life) later arrivals to the same
    instance (a release placed in that instance's FCFS stream)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pres = [gen_preload(rng, k, 32, 64, 10000, 0.7) for _ in range(n_instances)]
    t, times = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t > duration_s:
            break
        times.append(t)
    R = len(times)
    ranks = np.arange(1, n_instances + 1, dtype=np.float64)
    pz = ranks ** (-zipf_s)
    pz /= pz.sum()
    inst_of = rng.choice(n_instances, size=R, p=pz)
    per_inst: List[List[Dict[str, np.ndarray]]] = [[] for _ in range(n_instances)]
    local = np.zeros(R, np.int64)
    life = np.ceil(rng.exponential(mean_life, size=R)).astype(np.int64)
    for r in range(R):
        i = int(inst_of[r])
        local[r] = len(per_inst[i])
        per_inst[i].append(gen_request(rng, int(rng.integers(size_lo, size_hi + 1)), p_edge=0.1,
                                       bw=_bw_loguniform(1000.0)))
    insts = []
    for i in range(n_instances):
        n_i = len(per_inst[i])
        # FCFS stream: request j is released right after arrival j + life_j
        # of the same instance (if that arrival exists).
        lives = life[inst_of == i]
        rel_after: Dict[int, List[int]] = {}
        for j in range(n_i):
            a = j + int(lives[j])
            if a < n_i:
                rel_after.setdefault(a, []).append(j)
        ops: List[Tuple[int, int]] = []
        for j in range(n_i):
            ops.append((0, j))
            for jr in rel_after.get(j, []):
                ops.append((1, jr))
        insts.append(Instance(k, 32, 64, 10000, 6, method, pair_rule, WEIGHTS[6][scheme],
                              *pres[i], pack_requests(per_inst[i]), ops=ops))
    return Workload("serving", insts, np.asarray(times), inst_of.astype(np.int64), local)


def simulation(seed: int = 5, method: int = TOPSIS, pair_rule: int = RATIO,
               scheme: str = "flat", k: int = 20, n_requests: int = 6000, n_steps: int = 500,
               max_duration: int = 250, host_cpu: int = 24, host_mem: int = 256,
               link_mbps: int = 1000, n_criteria: int = 6):
    """The discrete-event scenario of the paper's GPU evaluation: an empty
    k-port fat-tree of host_cpu-core / host_mem-GB hosts and link_mbps links;
    n_requests of 4 containers (CPU U{1..2}, memory U{1..4}), up to half of a
    request's containers grouped in one pod, an Erdos-Renyi p=0.5 graph made
    connected with U{1..50} Mbps per link; submission step U{0..n_steps-1}
    and running time U{1..max_duration}.  Returns (workload, submit,
    duration)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for _ in range(n_requests):
        q = gen_request(rng, 4, p_edge=0.5, bw=lambda r, m: r.integers(1, 51, m), cpu_hi=2,
                        mem_hi=4)
        g = int(rng.integers(0, 3))  # containers grouped in pod 0 (0-2 of 4)
        if g >= 2:
            pod = np.concatenate([[0] * g, np.arange(1, 4 - g + 1)]).astype(np.int32)
            q["pod"] = pod
            # links inside the pod stay; pod ids are dense and ordered
        reqs.append(q)
    submit = np.sort(rng.integers(0, n_steps, n_requests)).astype(np.int32)
    duration = rng.integers(1, max_duration + 1, n_requests).astype(np.int32)
    W6 = WEIGHTS[n_criteria][scheme]
    inst = Instance(k, host_cpu, host_mem, link_mbps, n_criteria, method, pair_rule, W6,
                    None, None, None, pack_requests(reqs))
    return Workload("simulation", [inst]), submit, duration


def serving_events(wl: Workload):
    """Flattens a serving workload into one timed event list: each arrival
    (time, instance, kind 0, request index within the instance) followed by the
    departures its instance's FCFS stream places right after it (kind 1, with
    the event index of the departing request).  Returns arrays
    (t, inst, kind, local, release_of)."""
    t, inst, kind, local, rel = [], [], [], [], []
    ev_of = {}  # (instance, local request) -> event index
    pending = [dict() for _ in wl.instances]  # per instance: arrival j -> releases after it
    for i, ins in enumerate(wl.instances):
        last = None
        for k, r in ins.ops:
            if k == 0:
                last = r
            else:
                pending[i].setdefault(last, []).append(r)
    for g in range(len(wl.arrival_s)):
        i, j = int(wl.arrival_inst[g]), int(wl.arrival_local[g])
        ev_of[(i, j)] = len(t)
        t.append(float(wl.arrival_s[g])); inst.append(i); kind.append(0); local.append(j)
        rel.append(-1)
        for r in pending[i].get(j, []):
            t.append(float(wl.arrival_s[g])); inst.append(i); kind.append(1); local.append(r)
            rel.append(ev_of[(i, r)])
    return (np.asarray(t, np.float64), np.asarray(inst, np.int32), np.asarray(kind, np.int32),
            np.asarray(local, np.int32), np.asarray(rel, np.int32))


CONFIGS = {"small": small, "k16": k16, "k48": k48, "serving": serving, "batched": batched}

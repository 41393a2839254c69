#!/usr/bin/env python3
"""Benchmark of the GPU network-aware multi-criteria container scheduler.

Workload (default): 256 fat-tree data centers resident on the device, k
cycling over {8, 16, 24, 32} (819,200 hosts in total), each receiving 100
FCFS requests of 4-256 containers (singleton pods, Erdos-Renyi p=0.1 links,
log-uniform 1-1000 Mbps), 0-70 % random pre-load, TOPSIS over 6 criteria.
One step schedules every request of every instance from the pre-loaded
state, in one batched launch (one kernel per fat-tree size, one thread block
per data center) replayed from a CUDA graph.

Printed (rank 0, one JSON line): host-rankings/s of the whole job (pod
decisions x hosts ranked per decision), requests/s, p50/p99 request
completion latency inside the batched launch, the same work scheduled one
request per launch, the end-to-end rate through the C-ABI with host buffers,
the roofline of the scheduling kernel, the FP64 oracle timed on the host's
cores, and a serving replay (timed arrivals and departures through the
continuous-batching server, p50/p99 latency, against one request per launch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("host-rankings/sec and requests/sec (p50/p99 latency) at oracle-exact placements "
          "vs plain launch")
UNIT = "host-rankings/s"
BYTES_PER_HOST_RANKING = 16  # 4 int32 words of host state per host per decision
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--requests", type=int, default=100, help="requests per data center")
    ap.add_argument("--instances", type=int, default=256)
    ap.add_argument("--only-k", type=int, nargs="+", default=None,
                    help="keep only the data centers of these fat-tree sizes (the same "
                         "instances as in the full workload)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serving-events", type=int, default=0,
                    help="serving replay: leading timed events to replay (0 = all)")
    ap.add_argument("--serving-prefix", type=int, default=20000,
                    help="serving replay: leading events replayed by both arms (continuous "
                         "batching and one request per launch)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the one-request-per-launch run of the workload")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving replay (one JSON line); the default run starts it "
                         "as a child process so that it shares no device context with the "
                         "batched measurement")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (one block per data center)")
    ap.add_argument("--tune-ops", type=int, default=0,
                    help="operations per data center run in each autotuner trial (0: all; "
                         "a prefix of the chains can rank the shapes differently from the "
                         "whole chains, which set the batched makespan)")
    ap.add_argument("--no-largest", action="store_true",
                    help="skip the single k=48 data-center measurement")
    ap.add_argument("--largest-requests", type=int, default=200,
                    help="requests of the k=48 data center")
    ap.add_argument("--largest-shape", default="",
                    help="fixed launch shape BLOCKxBLOCKS_PER_DC for the k=48 data center "
                         "(default: autotuned)")
    ap.add_argument("--largest-only", action="store_true",
                    help="only the k=48 data-center measurement (one JSON line)")
    ap.add_argument("--no-largest-diff", action="store_true",
                    help="skip the k=48 AHP difference-rule measurement")
    ap.add_argument("--diff-requests", type=int, default=2,
                    help="requests of the k=48 AHP difference-rule data center")
    ap.add_argument("--diff-shape", default="1024x16",
                    help="launch shape BLOCKxBLOCKS_PER_DC of the k=48 AHP difference-rule run")
    ap.add_argument("--largest-diff-only", action="store_true",
                    help="only the k=48 AHP difference-rule measurement (one JSON line)")
    ap.add_argument("--no-comparators", action="store_true",
                    help="skip the method comparison (TOPSIS, AHP, best fit, worst fit)")
    ap.add_argument("--no-graph", action="store_true",
                    help="skip the general-graph widest-shortest-path measurement")
    ap.add_argument("--graph-pairs", type=int, default=2048)
    ap.add_argument("--no-simulation", action="store_true",
                    help="skip the discrete-event simulation with queueing")
    return ap.parse_args()


def workload(args, rank):
    from paper_1909_07673_gb300 import workloads as W
    wl = W.batched(seed=4 + 1000 * rank, n_instances=args.instances, n_requests=args.requests)
    if getattr(args, "only_k", None):
        wl = W.Workload(wl.name, [i for i in wl.instances if i.k in args.only_k])
        if not wl.instances:
            raise SystemExit("--only-k: no data center of those sizes")
    return wl


def config_dict(args, wl, world):
    hosts = sum(i.hosts for i in wl.instances)
    n = len(wl.instances)
    ks = "/".join(str(k) for k in sorted({i.k for i in wl.instances}))
    return {
        "workload": "batched fat-tree DCs: %d instances (k %s), %d requests of 4-256 "
                    "containers each, TOPSIS, 6 criteria" % (n, ks, args.requests),
        "instances_per_gpu": n,
        "requests_per_gpu": n * args.requests,
        "hosts_per_gpu": hosts,
        "method": "TOPSIS",
        "l2": "flushed before every step (256 MiB device write); request inputs exceed L2",
        "parallelism": "data centers sharded over %d rank(s), no collective" % world,
    }


# ----------------------------------------------------------------- oracle (CPU)

def oracle_sample(wl, seconds, threads=1):
    """Runs the FP64 oracle over whole FCFS chains (every request of a data
    center, so the sample covers every position in the chain) of the
    workload's data centers in their order (which cycles through the fat-tree
    sizes); each thread takes the next data center while less than `seconds`
    have passed and finishes the chain it started.  Returns (host_rankings,
    wall_s, description, requests, threads).  The oracle's C calls release
    the interpreter lock, so the threads run on separate cores."""
    import concurrent.futures as cf
    import oracle as O

    O.build_oracle()
    t0 = time.perf_counter()
    lock = threading.Lock()
    nxt = [0]
    tot = {"hr": 0, "reqs": 0, "inst": 0, "ks": {}}

    def worker():
        while time.perf_counter() - t0 < seconds:
            with lock:
                i = nxt[0]
                nxt[0] += 1
            if i >= len(wl.instances):
                return
            inst = wl.instances[i]
            dc = O.OracleDC.from_instance(inst)
            hr = 0
            for r in range(inst.reqs.n):
                out = dc.schedule(inst.reqs.request(r))
                hr += out["n_decisions"] * inst.hosts
            with lock:
                tot["hr"] += hr
                tot["reqs"] += inst.reqs.n
                tot["inst"] += 1
                tot["ks"][inst.k] = tot["ks"].get(inst.k, 0) + 1

    with cf.ThreadPoolExecutor(threads) as ex:
        for f in [ex.submit(worker) for _ in range(threads)]:
            f.result()
    wall = time.perf_counter() - t0
    ks = ", ".join("%d x k=%d" % (n, k) for k, n in sorted(tot["ks"].items()))
    desc = ("oracle.c (FP64), %d thread(s) over independent data centers: whole %d-request "
            "chains of %d data centers (%s), %.1f s" % (
                threads, wl.instances[0].reqs.n, tot["inst"], ks, wall))
    return tot["hr"], wall, desc, tot["reqs"], threads


def run_reference(args):
    """The reference arm: the FP64 oracle timed on the host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O

    O.build_oracle()
    wl = workload(args, 0)
    per = max(1.0, args.cpu_seconds / max(1, args.steps))
    times, hrs = [], []
    cores = os.cpu_count() or 1
    for s in range(args.warmup + args.steps):
        hr, wall, desc, reqs, _ = oracle_sample(wl, per, cores)
        if s >= args.warmup:
            times.append(wall)
            hrs.append(hr)
    value = sum(hrs) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, wl, 1),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step: " + desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- clocks

class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- helpers

def reduce_over_ranks(dist, times, counts, device):
    """Job-wide figures: the maximum of each time and the sum of each count
    over all ranks (dist None: one rank)."""
    import torch

    if dist is None:
        return [float(x) for x in times], [int(x) for x in counts]
    t = torch.tensor([float(x) for x in times] + [0.0], dtype=torch.float64, device=device)
    c = torch.tensor([int(x) for x in counts] + [0], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.tolist()[:-1]], [int(x) for x in c.tolist()[:-1]]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources that define the device code: every file under
    csrc/ except the host runtime (dc_runtime.cu: allocation, copies and
    launch bookkeeping, which the counters of a kernel do not depend on)."""
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1909_07673_gb300", "csrc", "*"))):
        if os.path.basename(f) == "dc_runtime.cu":
            continue
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_record():
    """The committed ncu record of the scheduling kernel (DRAM bytes, issue
    and pipe activity), or None when it is missing or was taken on other
    kernel sources."""
    p = os.path.join(ROOT, "profiles", "k_schedule_traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except Exception:
        return None
    return t if t.get("source_hash") == kernel_source_hash() else None


def ncu_traffic(host_rankings_per_launch):
    """DRAM bytes per launch of the scheduling kernel from the committed ncu
    record, scaled to this launch's host rankings; None without a record."""
    t = ncu_record()
    if t is None:
        return None
    return t["dram_bytes"] / t["host_rankings"] * host_rankings_per_launch


def ncu_pipes():
    """Issue and pipe activity of the dominant size class from the committed
    ncu record (fractions of peak on the SMs it runs on), or None."""
    t = ncu_record()
    if t is None or "issue_active_pct" not in t:
        return None
    return {"class": t["dominant_class"],
            "issue_active_frac": t["issue_active_pct"] / 100.0,
            "alu_pipe_frac": t["alu_pipe_active_pct"] / 100.0,
            "fmaheavy_pipe_frac": t["fmaheavy_pipe_active_pct"] / 100.0,
            "warp_instructions_per_host_ranking": t["warp_instructions_per_host_ranking"],
            "source": "profiles/k_schedule_traffic.json (ncu, same kernel sources)"}


# ----------------------------------------------------------------- serving

def run_serving(args, ds, torch):
    """Replays the serving workload (64 k=16 data centers, Poisson arrivals
    at 50k requests/s for 1 s, Zipf(1.1) over the data centers, 2-128
    containers, exponential lifetimes) through dc_server_replay: continuous
    batching and one request per launch on the same leading events
    (--serving-prefix), and continuous batching on all events.  Per data
    center: requests and p99 latency of the busiest ones (Zipf puts most of
    the load on a few), which attributes the tail."""
    from paper_1909_07673_gb300 import workloads as W

    wl = W.serving()
    ev = W.serving_events(wl)

    def replay(limit, per_launch):
        t, inst, kind, local, rel = (x[:limit] if limit else x for x in ev)
        reqs = [wl.instances[inst[e]].reqs.request(int(local[e])) if kind[e] == 0 else None
                for e in range(len(t))]
        dcs = [ds.DataCenter.from_instance(i, stream=torch.cuda.Stream()) for i in wl.instances]
        srv = ds.Server(dcs, admit_bytes=1 << 30, max_requests_per_launch=per_launch)
        lat, rid, st = srv.replay(t, inst, kind, reqs, rel)
        srv.close()
        for d in dcs:
            d.close()
        sub = kind == 0
        L = np.sort(lat[sub]) * 1e3
        per = []
        for i in np.argsort(-np.bincount(inst[sub], minlength=len(wl.instances)))[:3]:
            li = np.sort(lat[sub & (inst == i)]) * 1e3
            per.append({"instance": int(i), "requests": int(len(li)),
                        "p50_ms": float(li[len(li) // 2]) if len(li) else None,
                        "p99_ms": float(li[int(len(li) * 0.99)]) if len(li) else None})
        return {"events": int(len(t)), "requests": int(st["requests"]),
                "arrival_span_s": float(t[-1]), "wall_s": st["wall_s"],
                "requests_per_s": st["requests"] / st["wall_s"],
                "host_rankings_per_s": st["host_rankings"] / st["wall_s"],
                "launches": int(st["launches"]),
                "latency_ms": {"p50": float(L[len(L) // 2]), "p99": float(L[int(len(L) * 0.99)])},
                "busiest_instances": per}

    n = args.serving_prefix
    return {
        "workload": "64 k=16 data centers (0-70 %% pre-load), Poisson %d requests/s for 1 s, "
                    "Zipf(1.1) over data centers, 2-128 containers, lifetimes Exp(100 arrivals)"
                    % 50000,
        "latency": "arrival (replayed on the host clock) to completion seen by the host",
        "same_prefix": {"events": n,
                        "continuous_batching": replay(n, 0),
                        "plain_launch": dict(replay(n, 1),
                                             note="one request per launch, one launch at a time")},
        "continuous_batching_all_events": replay(args.serving_events, 0),
    }


# ----------------------------------------------------------------- method comparison

def run_comparators(args, ds, torch):
    """The k=16 workload's requests (1,000 of 4-64 containers, [min, max]
    intervals) on an empty k=16 fat-tree, scheduled by TOPSIS, AHP and the
    best-fit / worst-fit comparators: device time, acceptance, mean utilities
    (Eqs. 1-2) and the final fragmentation."""
    from paper_1909_07673_gb300 import workloads as W

    out = {}
    stream = torch.cuda.Stream()
    for name, method in (("TOPSIS", W.TOPSIS), ("AHP", W.AHP), ("BF", W.BF), ("WF", W.WF)):
        inst = W.k16(method=method, intervals=True, preload=0.0).instances[0]
        dc = ds.load_instance(inst, stream=stream)
        plan = ds.Plan([dc], ds.PLAN_RESET)
        times = []
        for rep in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.launch(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                times.append(e0.elapsed_time(e1))
        plan.collect()
        dec, hr, _, _ = plan.stats()
        ms = statistics.mean(times)
        acc = sum(dc.status(r)[0] == ds.ACCEPTED for r in range(inst.reqs.n))
        u = dc.utility_summary()
        act_s, act_l, f_s, f_l = dc.fragmentation()
        out[name] = {
            "ms_per_launch": ms, "decisions": dec, "host_rankings_per_s": hr / (ms * 1e-3),
            "accepted_requests": int(acc),
            "mean_u_container": u["sum_u_container"] / max(1, u["n_containers"]),
            "mean_u_link": u["sum_u_link"] / max(1, u["n_links"]),
            "f_servers": f_s, "f_links": f_l,
        }
        plan.close()
        dc.close()
    return {"workload": "one empty k=16 fat-tree (1,024 hosts), 1,000 requests of 4-64 "
                        "containers with [min, max] intervals, 6 criteria",
            "methods": out}


# ----------------------------------------------------------------- simulation

def run_simulation(args, ds, torch):
    """The discrete-event simulation with queueing (dc_simulate, one launch
    per run) on the GPU evaluation's scenario (k=20 fat-tree of 24-core /
    256 GB hosts, 1 Gbps, 6,000 four-container requests over 500 steps,
    running times up to 250) and on a loaded one (k=8 of 8-core / 16 GB hosts,
    200 Mbps, 2,000 requests), for TOPSIS, AHP, best fit and worst fit: wall
    time of the call, requests started, queueing delay (steps), decisions;
    the oracle timed on the first scenario with TOPSIS."""
    import oracle as O
    from paper_1909_07673_gb300 import workloads as W

    scen = {"paper_k20": dict(k=20, n_requests=6000, n_steps=500, max_duration=250),
            "loaded_k8": dict(k=8, n_requests=2000, n_steps=500, max_duration=250,
                              host_cpu=8, host_mem=16, link_mbps=200)}
    out = {}
    stream = torch.cuda.Stream()
    for name, cfg in scen.items():
        out[name] = {"config": cfg, "methods": {}}
        for mname, m in (("TOPSIS", W.TOPSIS), ("AHP", W.AHP), ("BF", W.BF), ("WF", W.WF)):
            wl, sub, dur = W.simulation(method=m, **cfg)
            inst = wl.instances[0]
            dc = ds.load_instance(inst, stream=stream)
            torch.cuda.synchronize()
            t = time.perf_counter()
            start = dc.simulate(cfg["n_steps"], sub, dur)
            sec = time.perf_counter() - t
            st = start >= 0
            delay = (start - sub)[st]
            dec = sum(dc.status(r)[1] for r in range(inst.reqs.n))
            out[name]["methods"][mname] = {
                "wall_s": sec, "started": int(st.sum()), "requests": int(inst.reqs.n),
                "delay_mean": float(delay.mean()) if len(delay) else None,
                "delay_p99": float(np.percentile(delay, 99)) if len(delay) else None,
                "decisions": int(dec), "us_per_decision": sec * 1e6 / max(1, dec)}
            dc.close()
    wl, sub, dur = W.simulation(method=W.TOPSIS, **scen["paper_k20"])
    inst = wl.instances[0]
    odc = O.OracleDC.from_instance(inst)
    t = time.perf_counter()
    odc.simulate([inst.reqs.request(r) for r in range(inst.reqs.n)], sub, dur, 500)
    out["paper_k20"]["oracle_topsis_s"] = time.perf_counter() - t
    return out


# ----------------------------------------------------------------- general graphs

def run_graph_paths(args, ds, torch, peak):
    """Widest shortest paths between random host pairs of the k=48 fat-tree
    taken as a general graph (30,528 nodes, 82,944 links, residuals
    U[0, 1) x 40 Gbps pre-load), through dc_graph_widest_paths (host arrays
    in and out); the oracle's search timed on a sample of the pairs."""
    import oracle as O

    k, H = 48, 48 ** 3 // 4
    rng = np.random.default_rng(48)
    res = (40000 - np.floor(rng.random(3 * H) * 40000)).astype(np.int32)
    V, lu, lv = O.fattree_graph(k, res)
    pairs = rng.integers(0, H, (args.graph_pairs, 2)).astype(np.int32)
    g = ds.Graph(V, lu, lv, res)
    g.widest_paths(pairs[:64, 0], pairs[:64, 1], 8)  # warm-up
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        hops, bott, links = g.widest_paths(pairs[:, 0], pairs[:, 1], 8)
        times.append(time.perf_counter() - t)
    g.close()
    sec = min(times)
    # algorithmic bytes of one pair: two breadth-first passes, each reading
    # every adjacency entry (neighbour, link, residual, label: 16 B) and
    # writing / reading every node's two labels and queue slot (16 B)
    bytes_pair = 2 * (16 * 2 * len(lu) + 16 * V)
    gbs = args.graph_pairs * bytes_pair / sec / 1e9
    og = O.OracleGraph(V, lu, lv, res)
    t = time.perf_counter()
    n_or = 0
    while n_or < args.graph_pairs and time.perf_counter() - t < 5.0:
        og.widest_path(int(pairs[n_or, 0]), int(pairs[n_or, 1]))
        n_or += 1
    osec = time.perf_counter() - t
    return {
        "workload": "k=48 fat-tree as a general graph (%d nodes, %d links), %d random host "
                    "pairs" % (V, len(lu), args.graph_pairs),
        "pairs_per_s": args.graph_pairs / sec, "ms_per_call": sec * 1e3,
        "note": "wall time of dc_graph_widest_paths (pairs in, hops / bottleneck / links "
                "out through host memory)",
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak, "bytes_per_pair": bytes_pair},
        "cpu_oracle": {"pairs_per_s": n_or / osec, "cores": 1,
                       "sample": "first %d pairs, one thread" % n_or},
    }


# ----------------------------------------------------------------- largest fat-tree

def run_largest(args, ds, torch, peak):
    """One k=48 data center (27,648 hosts, 40 Gbps, 0-100 % pre-load), 200
    requests of 64-512 containers in pods of 1-8, Pareto bandwidths, TOPSIS
    over 6 criteria: a single sequential chain of pod decisions, scheduled
    with the autotuned cluster shape (state-resetting launches)."""
    from paper_1909_07673_gb300 import workloads as W

    inst = W.k48().instances[0]
    stream = torch.cuda.Stream()
    dc = ds.load_instance(inst, stream=stream, max_requests=args.largest_requests)
    tuned = None
    if args.largest_shape:
        b, n = (int(x) for x in args.largest_shape.lower().split("x"))
        ds.set_launch(inst.k, inst.n_criteria, inst.method, inst.pair_rule, b, n)
    elif not args.no_autotune:
        tuned = ds.autotune([dc], max_ops=8)
    plan = ds.Plan([dc], ds.PLAN_RESET)
    times = []
    for rep in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.launch(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e1))
    plan.collect()
    dec, hr, nk, _ = plan.stats()
    ms = statistics.mean(times)
    block, ncta, _ = ds.get_launch(dc)
    acc = sum(dc.status(r)[0] == ds.ACCEPTED for r in range(min(inst.reqs.n, args.largest_requests)))
    gbs = hr * BYTES_PER_HOST_RANKING / (ms * 1e-3) / 1e9
    plan.close()
    dc.close()
    return {
        "workload": "one k=48 fat-tree (27,648 hosts), %d requests of 64-512 containers in "
                    "pods of 1-8, TOPSIS, 6 criteria" % min(inst.reqs.n, args.largest_requests),
        "host_rankings_per_s": hr / (ms * 1e-3), "decisions_per_s": dec / (ms * 1e-3),
        "us_per_decision": ms * 1e3 / dec, "ms_per_launch": ms, "decisions": dec,
        "accepted_requests": int(acc),
        "launch_shape": {"block": block, "blocks_per_dc": ncta,
                         "trials": tuned[0]["trials"] if tuned else 0},
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                     "frac": gbs / peak,
                     "note": "16 B of host state per host ranking; one data center is a "
                             "sequential chain of decisions (latency-bound)"},
    }


# ----------------------------------------------------------------- AHP DIFF

SM_COUNT = 152
LANES_PER_SM = 128  # FP32 lanes per SM


def run_largest_diff(args, ds, torch):
    """AHP with the difference rule on one k=48 data center at the paper's
    scale (27,648 hosts, 40 Gbps links, 0-100 % pre-load), the first
    --diff-requests requests of the k48 workload (64-512 containers in pods
    of 1-8), on one thread-block cluster (state-resetting launches, CUDA
    events).  The work is the definition's: per decision and criterion, the
    pairwise column and row sums over the D_v distinct values of the viable
    hosts, 2 D_v^2 pair evaluations (the kernel counts them); ALU roofline
    with 4 operations per pair evaluation (difference, comparison /
    selection, reciprocal, accumulation) against the FP32 lanes of the whole
    GPU at the sampled clock."""
    from paper_1909_07673_gb300 import workloads as W

    inst = W.k48(n_requests=args.diff_requests, method=W.AHP, pair_rule=W.DIFF).instances[0]
    stream = torch.cuda.Stream()
    b, n = (int(x) for x in args.diff_shape.lower().split("x"))
    ds.set_launch(inst.k, inst.n_criteria, inst.method, inst.pair_rule, b, n)
    try:
        dc = ds.load_instance(inst, stream=stream)
        plan = ds.Plan([dc], ds.PLAN_RESET)
        times = []
        with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            for rep in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plan.launch(stream)
                e1.record(stream)
                torch.cuda.synchronize()
                if rep > 0:
                    times.append(e0.elapsed_time(e1))
        plan.collect()
        dec, hr, _, _ = plan.stats()
        pairs = plan.diff_pairs()
        block, ncta, _ = ds.get_launch(dc)
        acc = sum(dc.status(r)[0] == ds.ACCEPTED for r in range(inst.reqs.n))
        plan.close()
        dc.close()
    finally:
        ds.set_launch(inst.k, inst.n_criteria, inst.method, inst.pair_rule, 0, 1)
    ms = statistics.mean(times)
    ck = clk.summary()
    mhz = ck.get("sm_mhz") or 2070.0
    peak = SM_COUNT * LANES_PER_SM * mhz * 1e6 / 1e12
    achieved = 4.0 * pairs / (ms * 1e-3) / 1e12
    return {
        "workload": "one k=48 fat-tree (27,648 hosts, 40 Gbps), first %d requests of 64-512 "
                    "containers in pods of 1-8, AHP difference rule, 6 criteria" % inst.reqs.n,
        "launch_shape": {"block": block, "blocks_per_dc": ncta},
        "ms_per_launch": ms, "decisions": dec, "us_per_decision": ms * 1e3 / max(1, dec),
        "host_rankings_per_s": hr / (ms * 1e-3), "accepted_requests": int(acc),
        "pair_evaluations": pairs, "pair_evaluations_per_s": pairs / (ms * 1e-3),
        "pair_evaluations_per_decision": pairs / max(1, dec),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak,
                     "note": "4 ops per pair evaluation x 2 sum_v D_v^2 pairs per decision; peak "
                             "= %d SMs x %d FP32 lanes x %.0f MHz (sampled); the data center "
                             "runs on %d of the %d SMs" % (SM_COUNT, LANES_PER_SM, mhz, ncta,
                                                           SM_COUNT)},
        "clocks": ck,
    }


# ----------------------------------------------------------------- ours

def run_largest_diff_only(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__

    __graft_entry__.build()
    from paper_1909_07673_gb300 import dcsched as ds

    print(json.dumps({"largest_fat_tree_diff": run_largest_diff(args, ds, torch)}), flush=True)
    return 0


def run_largest_only(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__

    __graft_entry__.build()
    from paper_1909_07673_gb300 import dcsched as ds

    peak, _ = measured_peak()
    print(json.dumps({"largest_fat_tree": run_largest(args, ds, torch, peak)}), flush=True)
    return 0


def run_serving_only(args):
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import __graft_entry__

    __graft_entry__.build()
    from paper_1909_07673_gb300 import dcsched as ds

    print(json.dumps({"serving": run_serving(args, ds, torch)}), flush=True)
    return 0


def serving_child(args):
    """The serving replay in a child process on this rank's GPU (nothing
    else runs on the device meanwhile); its JSON result."""
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "WORLD_SIZE", "LOCAL_WORLD_SIZE", "GROUP_RANK")}
    cmd = [sys.executable, os.path.abspath(__file__), "--serving-only",
           "--serving-events", str(args.serving_events), "--serving-prefix",
           str(args.serving_prefix)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("serving replay failed:\n" + r.stderr[-4000:])
    return json.loads(r.stdout.strip().splitlines()[-1])["serving"]


def run_plain(args, ds, wl, stream):
    """The workload scheduled one request per launch (see run_ours)."""
    dcs = [ds.DataCenter.from_instance(inst, stream=stream) for inst in wl.instances]
    R = max(inst.reqs.n for inst in wl.instances)
    lat, hr, n = [], 0, 0
    t0 = time.perf_counter()
    for r in range(R):
        for dc, inst in zip(dcs, wl.instances):
            if r >= inst.reqs.n:
                continue
            dc.submit(inst.reqs.request(r))
            ds.schedule([dc])
            st, nd, _ = dc.status(r)
            lat.append(time.perf_counter() - t0)
            hr += nd * inst.hosts
            n += 1
    wall = time.perf_counter() - t0
    for dc in dcs:
        dc.close()
    lat = np.sort(np.array(lat)) * 1e3
    return {"requests": n, "wall_s": wall, "requests_per_s": n / wall,
            "host_rankings_per_s": hr / wall,
            "latency_ms": {"p50": float(lat[len(lat) // 2]), "p99": float(lat[int(len(lat) * 0.99)])},
            "note": "every request of the workload, one request per launch (submit, schedule, "
                    "synchronize, read), round-robin over the data centers; latency = completion "
                    "time from the start (all requests arrive at the start, as for the batched "
                    "launch)"}


def optional_section(name, fn, *a):
    """Runs a section reported beside the main measurement; a failure is
    reported in that section's key ({"error": ...}, also on stderr) instead of
    costing the whole JSON line."""
    try:
        return fn(*a)
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        print("bench: section %s failed: %r" % (name, e), file=sys.stderr, flush=True)
        return {"error": "%s: %s" % (type(e).__name__, str(e)[-2000:])}


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    from paper_1909_07673_gb300 import dcsched as ds

    # the serving replay first, on an otherwise idle device (rank 0), in a
    # process of its own: run in this process before the autotuner, it left
    # the batched step ~7% slower (measured; each alone did not)
    serving = None if (args.no_serving or rank != 0) else optional_section(
        "serving", serving_child, args)
    if dist:
        dist.barrier()
    wl = workload(args, rank)
    stream = torch.cuda.Stream()
    dcs = [ds.load_instance(inst, stream=stream) for inst in wl.instances]
    tuned = None if args.no_autotune else ds.autotune(dcs, max_ops=args.tune_ops)
    plan = ds.Plan(dcs, ds.PLAN_GRAPH | ds.PLAN_RESET)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step():
        with torch.cuda.stream(stream):
            flush.zero_()
        plan.launch(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[i][0].record(stream)
            plan.launch(stream)
            ev[i][1].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    ms_step = t0.elapsed_time(t1) / args.steps
    ms_kernel = statistics.mean(a.elapsed_time(b) for a, b in ev)
    plan.collect()
    dec, hr, nkern, start_ns = plan.stats()
    n_req = sum(inst.reqs.n for inst in wl.instances)
    lat = []
    accepted = 0
    for dc, inst in zip(dcs, wl.instances):
        for r in range(inst.reqs.n):
            st, nd, done = dc.status(r)
            lat.append((done - start_ns) * 1e-6)
            accepted += st == ds.ACCEPTED
    (ms_step, ms_kernel), (hr_all, dec_all, req_all, acc_all) = reduce_over_ranks(
        dist, [ms_step, ms_kernel], [hr, dec, n_req, accepted], "cuda")

    # one request per launch on the same workload: every request of every
    # data center arrives at the start, and each is submitted, scheduled alone
    # (one launch) and read back before the next; round-robin over the data
    # centers, each data center's requests in FCFS order; latency = completion
    # time from the start, as for the batched launch
    plain = None if args.no_plain else run_plain(args, ds, wl, stream)

    # end to end through the C-ABI with host buffers: submit every request
    # (host copies; the data centers are independent, so a pool of host
    # threads packs them, one data center per task, the library call
    # releasing the interpreter lock), schedule (inputs host->device,
    # kernels, results device->host), read a result
    from concurrent.futures import ThreadPoolExecutor
    from paper_1909_07673_gb300.dcsched import _Req, _Request, lib as _lib
    batches = []
    for inst in wl.instances:
        reqs = [_Req(inst.reqs.request(r)) for r in range(inst.reqs.n)]
        batches.append((reqs, (_Request * len(reqs))(*[q.s for q in reqs])))
    n_submit = max(1, min(len(dcs), os.cpu_count() or 1))

    def submit_all(job):
        dc, (reqs, arr) = job
        ds._check(_lib().dc_reset(dc.h), "dc_reset")
        ds._check(_lib().dc_submit_batch(dc.h, len(reqs), arr, None), "dc_submit_batch")

    pool = ThreadPoolExecutor(max_workers=n_submit)
    io0 = [dc.io_stats() for dc in dcs]
    e2e_times = []
    for s in range(1 + args.e2e_steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        list(pool.map(submit_all, zip(dcs, batches)))
        ds.schedule(dcs)
        dcs[0].status(0)
        if s > 0:
            e2e_times.append(time.perf_counter() - t)
        else:
            io0 = [dc.io_stats() for dc in dcs]
    pool.shutdown()
    io1 = [dc.io_stats() for dc in dcs]
    h2d = sum(b[0] - a[0] for a, b in zip(io0, io1)) / args.e2e_steps
    d2h = sum(b[1] - a[1] for a, b in zip(io0, io1)) / args.e2e_steps
    (e2e_s,), _ = reduce_over_ranks(dist, [statistics.mean(e2e_times)], [], "cuda")
    e2e_value = hr_all / e2e_s

    peak, peak_kind = measured_peak()
    achieved = hr * BYTES_PER_HOST_RANKING / (ms_kernel * 1e-3) / 1e9
    traffic = ncu_traffic(hr)
    largest = None if args.no_largest else optional_section(
        "largest_fat_tree", run_largest, args, ds, torch, peak)
    largest_diff = None if (args.no_largest_diff or rank != 0) else optional_section(
        "largest_fat_tree_diff", run_largest_diff, args, ds, torch)
    comparators = None if (args.no_comparators or rank != 0) else optional_section(
        "comparators", run_comparators, args, ds, torch)
    graph = None if (args.no_graph or rank != 0) else optional_section(
        "graph_paths", run_graph_paths, args, ds, torch, peak)
    simulation = None if (args.no_simulation or rank != 0) else optional_section(
        "simulation", run_simulation, args, ds, torch)
    if rank != 0:
        if dist:
            dist.barrier()
        return 0
    cpu_hr, cpu_s, cpu_desc, _, cpu_threads = oracle_sample(wl, args.cpu_seconds,
                                                            os.cpu_count() or 1)
    one_hr, one_s, one_desc, _, _ = oracle_sample(wl, max(2.0, args.cpu_seconds / 3), 1)
    lat.sort()
    cfg = config_dict(args, wl, world)
    if tuned is not None:
        cfg["launch_shapes"] = [
            {"k": e["k"], "block": e["block"], "blocks_per_dc": e["ncta"],
             "default": [e["block0"], e["ncta0"]], "trials": e["trials"],
             "kept_after_full_check": e["kept"]} for e in tuned]
        cfg["autotune"] = (
            "coordinate descent over launch shapes per fat-tree size, each trial a "
            "state-resetting launch of all operations of every data center (the timed "
            "step's work)" if args.tune_ops <= 0 else
            "coordinate descent over launch shapes per fat-tree size, each trial a "
            "state-resetting launch of the first %d operations of every data center; the "
            "result is kept only if faster than the starting shapes on all operations"
            % args.tune_ops)
    line = {
        "metric": METRIC, "value": hr_all / (ms_step * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "host_rankings_per_step": hr_all, "decisions_per_step": dec_all,
        "requests_per_s": req_all / (ms_step * 1e-3),
        "decisions_per_s": dec_all / (ms_step * 1e-3),
        "accepted_fraction": acc_all / req_all,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[int(len(lat) * 0.99)],
                       "note": "request completion time from the start of the batched launch"},
        "plain_launch": plain,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "submit_threads": n_submit},
        "gpu_launches": args.steps * nkern,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind + " (STREAM-style copy)",
                     "pipes": ncu_pipes(),
                     "note": "16 B of host state per host ranking over the scheduling launch "
                             "(graph: state reset + one kernel per fat-tree size)"},
        "cpu_baseline": {"value": cpu_hr / cpu_s, "unit": UNIT, "cores": cpu_threads,
                         "kind": "oracle", "sample": cpu_desc,
                         "single_thread": {"value": one_hr / one_s, "sample": one_desc}},
        "clocks": clk.summary(),
    }
    if serving is not None:
        line["serving"] = serving
    if largest is not None:
        line["largest_fat_tree"] = largest
    if largest_diff is not None:
        line["largest_fat_tree_diff"] = largest_diff
    if comparators is not None:
        line["comparators"] = comparators
    if graph is not None:
        line["graph_paths"] = graph
    if simulation is not None:
        line["simulation"] = simulation
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.largest_only:
        return run_largest_only(args)
    if args.largest_diff_only:
        return run_largest_diff_only(args)
    if args.serving_only:
        return run_serving_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

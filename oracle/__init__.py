"""ctypes binding of the FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the CPU-baseline leg of bench.py.  The CUDA library and its Python binding
never import this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TOPSIS, AHP, BF, WF = 0, 1, 2, 3
RATIO, DIFF = 0, 1
ACCEPTED, REJECTED = 1, 2
FREE_CPU, FREE_MEM, CTR, PRE, LINK_RES = 0, 1, 2, 3, 4

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)


def build_oracle(force: bool = False) -> str:
    """Compiles oracle.c into liboracle.so next to it (plain gcc, FP64,
    no floating-point contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Config(C.Structure):
    _fields_ = [("k", C.c_int32), ("host_cpu", C.c_int32), ("host_mem", C.c_int32),
                ("link_mbps", C.c_int32), ("n_criteria", C.c_int32), ("method", C.c_int32),
                ("pair_rule", C.c_int32), ("weights", C.c_double * 6)]


class _Request(C.Structure):
    _fields_ = [("n_containers", C.c_int32), ("n_edges", C.c_int32),
                ("cpu_min", _i32p), ("cpu_max", _i32p), ("mem_min", _i32p),
                ("mem_max", _i32p), ("pod", _i32p), ("src", _i32p), ("dst", _i32p),
                ("bw_min", _i32p), ("bw_max", _i32p)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_decisions", C.c_int32), ("host", _i32p),
                ("cpu", _i32p), ("mem", _i32p), ("bw", _i32p), ("path", _i32p),
                ("pod_score", _f64p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        L = _lib
        L.orc_fattree_dims.argtypes = [C.c_int32] + [_i64p] * 5
        L.orc_create.argtypes = [C.POINTER(_Config), _i32p, _i32p, _i32p, C.POINTER(C.c_void_p)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_schedule.argtypes = [C.c_void_p, C.POINTER(_Request), C.POINTER(_Result)]
        L.orc_release.argtypes = [C.c_void_p, C.POINTER(_Request), C.POINTER(_Result)]
        L.orc_get_state.argtypes = [C.c_void_p, C.c_int32, _i32p, C.c_int64]
        L.orc_set_state.argtypes = [C.c_void_p, C.c_int32, _i32p, C.c_int64]
        L.orc_widest_path.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _i32p, _i32p]
        L.orc_widest_path.restype = C.c_int32
        L.orc_rank_pod.argtypes = [C.c_void_p, C.POINTER(_Request), C.c_int32, _i32p, _i32p,
                                   _i64p, _f64p]
        L.orc_rank_pod.restype = C.c_int32
        L.orc_topsis.argtypes = [C.c_int32, C.c_int32, _i64p, _f64p, _f64p]
        L.orc_ahp_weights.argtypes = [C.c_int32, _f64p, C.c_int32, _f64p]
        L.orc_ahp.argtypes = [C.c_int32, C.c_int32, _i64p, _f64p, C.c_int32, _f64p]
        L.orc_ahp_literal.argtypes = [C.c_int32, C.c_int32, _i64p, _f64p, C.c_int32, _f64p]
        L.orc_utilities.argtypes = [C.POINTER(_Request), C.POINTER(_Result), _f64p, _f64p]
        L.orc_utilities.restype = None
        L.orc_fragmentation.argtypes = [C.c_void_p, _i64p, _i64p, _f64p, _f64p]
        L.orc_fragmentation.restype = None
        L.orc_simulate.argtypes = [C.c_void_p, C.c_int32, C.POINTER(_Request), _i32p, _i32p,
                                   C.c_int32, C.POINTER(_Result), _i32p]
        L.orc_graph_create.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, _i32p,
                                       C.POINTER(C.c_void_p)]
        L.orc_graph_destroy.argtypes = [C.c_void_p]
        L.orc_graph_destroy.restype = None
        L.orc_graph_widest_path.argtypes = [C.c_void_p, C.c_int32, C.c_int32, _i32p, _i32p,
                                            _i32p, C.c_int32]
        L.orc_graph_widest_path.restype = C.c_int32
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def fattree_dims(k: int) -> Dict[str, int]:
    v = [C.c_int64() for _ in range(5)]
    rc = lib().orc_fattree_dims(k, *[C.byref(x) for x in v])
    if rc != 0:
        raise ValueError("invalid k")
    return dict(zip(("hosts", "edge", "agg", "core", "links"), (x.value for x in v)))


def _weights6(w: Sequence[float]):
    arr = (C.c_double * 6)()
    for i, x in enumerate(w):
        arr[i] = float(x)
    return arr


class _Req:
    """Keeps the numpy arrays of a request alive for the ctypes struct."""

    def __init__(self, q: Dict[str, np.ndarray]):
        self.a = {k: np.ascontiguousarray(v, np.int32) for k, v in q.items()}
        a = self.a
        self.s = _Request(len(a["pod"]), len(a["src"]), *(
            _p(a[n], _i32p) for n in ("cpu_min", "cpu_max", "mem_min", "mem_max", "pod",
                                      "src", "dst", "bw_min", "bw_max")))
        self.n_pods = int(a["pod"].max()) + 1 if len(a["pod"]) else 0


class OracleDC:
    def __init__(self, k, host_cpu, host_mem, link_mbps, n_criteria, method, pair_rule,
                 weights, pre_cpu=None, pre_mem=None, pre_link=None):
        self.cfg = _Config(k, host_cpu, host_mem, link_mbps, n_criteria, method, pair_rule,
                           _weights6(weights))
        self.k = k
        self.H = k ** 3 // 4
        self.n_criteria = n_criteria
        pc = None if pre_cpu is None else np.ascontiguousarray(pre_cpu, np.int32)
        pm = None if pre_mem is None else np.ascontiguousarray(pre_mem, np.int32)
        pl = None if pre_link is None else np.ascontiguousarray(pre_link, np.int32)
        h = C.c_void_p()
        rc = lib().orc_create(C.byref(self.cfg), None if pc is None else _p(pc, _i32p),
                              None if pm is None else _p(pm, _i32p),
                              None if pl is None else _p(pl, _i32p), C.byref(h))
        if rc != 0:
            raise ValueError("orc_create failed: %d" % rc)
        self.h = h

    @classmethod
    def from_instance(cls, inst) -> "OracleDC":
        return cls(inst.k, inst.host_cpu, inst.host_mem, inst.link_mbps, inst.n_criteria,
                   inst.method, inst.pair_rule, inst.weights, inst.pre_cpu, inst.pre_mem,
                   inst.pre_link)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_destroy(self.h)
            self.h = None

    def schedule(self, q: Dict[str, np.ndarray]) -> Dict[str, np.ndarray]:
        rq = _Req(q)
        n, m, P = len(rq.a["pod"]), len(rq.a["src"]), rq.n_pods
        out = {"host": np.zeros(n, np.int32), "cpu": np.zeros(n, np.int32),
               "mem": np.zeros(n, np.int32), "bw": np.zeros(m, np.int32),
               "path": np.zeros(6 * m, np.int32), "pod_score": np.zeros(P, np.float64)}
        res = _Result(0, 0, *(_p(out[x], _i32p) for x in ("host", "cpu", "mem", "bw", "path")),
                      _p(out["pod_score"], _f64p))
        rc = lib().orc_schedule(self.h, C.byref(rq.s), C.byref(res))
        if rc != 0:
            raise ValueError("orc_schedule failed: %d" % rc)
        out["status"] = int(res.status)
        out["n_decisions"] = int(res.n_decisions)
        return out

    def release(self, q: Dict[str, np.ndarray], out: Dict[str, np.ndarray]) -> None:
        rq = _Req(q)
        res = _Result(out["status"], out["n_decisions"],
                      *(_p(out[x], _i32p) for x in ("host", "cpu", "mem", "bw", "path")),
                      _p(out["pod_score"], _f64p))
        rc = lib().orc_release(self.h, C.byref(rq.s), C.byref(res))
        if rc != 0:
            raise ValueError("orc_release failed: %d" % rc)

    def state(self, field: int) -> np.ndarray:
        n = 3 * self.H if field == LINK_RES else self.H
        a = np.zeros(n, np.int32)
        if lib().orc_get_state(self.h, field, _p(a, _i32p), n) != 0:
            raise ValueError("bad field")
        return a

    def set_state(self, field: int, a: np.ndarray) -> None:
        a = np.ascontiguousarray(a, np.int32)
        if lib().orc_set_state(self.h, field, _p(a, _i32p), len(a)) != 0:
            raise ValueError("bad field")

    def simulate(self, reqs, submit, duration, n_steps: int):
        """Discrete-event simulation with queueing over the requests (orc_simulate):
        returns (results, start steps)."""
        keep = [_Req(q) for q in reqs]
        n = len(keep)
        arr = (_Request * max(1, n))(*[k.s for k in keep])
        outs, res = [], (_Result * max(1, n))()
        for i, k in enumerate(keep):
            nc, m, P = len(k.a["pod"]), len(k.a["src"]), k.n_pods
            o = {"host": np.zeros(nc, np.int32), "cpu": np.zeros(nc, np.int32),
                 "mem": np.zeros(nc, np.int32), "bw": np.zeros(m, np.int32),
                 "path": np.zeros(6 * m, np.int32), "pod_score": np.zeros(P, np.float64)}
            outs.append(o)
            res[i] = _Result(0, 0, *(_p(o[x], _i32p) for x in ("host", "cpu", "mem", "bw", "path")),
                             _p(o["pod_score"], _f64p))
        sub = np.ascontiguousarray(submit, np.int32)
        dur = np.ascontiguousarray(duration, np.int32)
        start = np.zeros(max(1, n), np.int32)
        rc = lib().orc_simulate(self.h, n, arr, _p(sub, _i32p), _p(dur, _i32p), int(n_steps), res,
                                _p(start, _i32p))
        if rc != 0:
            raise ValueError("orc_simulate failed: %d" % rc)
        for i, o in enumerate(outs):
            o["status"] = int(res[i].status)
            o["n_decisions"] = int(res[i].n_decisions)
        return outs, start[:n]

    def fragmentation(self):
        """(active servers, active links, F(N^s), F(E^s)) of the current state."""
        a, b = C.c_int64(), C.c_int64()
        fs, fl = C.c_double(), C.c_double()
        lib().orc_fragmentation(self.h, C.byref(a), C.byref(b), C.byref(fs), C.byref(fl))
        return a.value, b.value, fs.value, fl.value

    def widest_path(self, u: int, v: int):
        links = np.zeros(6, np.int32)
        hops = C.c_int32()
        b = lib().orc_widest_path(self.h, u, v, _p(links, _i32p), C.byref(hops))
        return int(b), links, int(hops.value)

    def rank_pod(self, q: Dict[str, np.ndarray], g: int, host_of: np.ndarray):
        rq = _Req(q)
        ho = np.ascontiguousarray(host_of, np.int32)
        feas = np.zeros(self.H, np.int32)
        crit = np.zeros(self.H * self.n_criteria, np.int64)
        score = np.zeros(self.H, np.float64)
        F = lib().orc_rank_pod(self.h, C.byref(rq.s), g, _p(ho, _i32p), _p(feas, _i32p),
                               _p(crit, _i64p), _p(score, _f64p))
        if F < 0:
            raise ValueError("orc_rank_pod failed: %d" % F)
        return feas.astype(bool), crit.reshape(self.H, self.n_criteria), score


class OracleGraph:
    """Undirected graph with per-link residual bandwidth (orc_graph)."""

    def __init__(self, n_nodes: int, lu, lv, res):
        self.V = int(n_nodes)
        self.lu = np.ascontiguousarray(lu, np.int32)
        self.lv = np.ascontiguousarray(lv, np.int32)
        self.res = np.ascontiguousarray(res, np.int32)
        h = C.c_void_p()
        rc = lib().orc_graph_create(self.V, len(self.lu), _p(self.lu, _i32p), _p(self.lv, _i32p),
                                    _p(self.res, _i32p), C.byref(h))
        if rc != 0:
            raise ValueError("orc_graph_create failed: %d" % rc)
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_graph_destroy(self.h)
            self.h = None

    def widest_path(self, s: int, t: int, max_nodes: int = 64):
        """(hops, bottleneck, nodes, links); hops -1 when unreachable."""
        b = C.c_int32()
        nodes = np.full(max_nodes, -1, np.int32)
        links = np.full(max_nodes, -1, np.int32)
        h = lib().orc_graph_widest_path(self.h, s, t, C.byref(b), _p(nodes, _i32p),
                                        _p(links, _i32p), max_nodes)
        if h < 0:
            return -1, -1, nodes[:0], links[:0]
        return h, b.value, nodes[:h + 1], links[:h]


def fattree_graph(k: int, res):
    """A k-port fat-tree as a general graph: nodes hosts [0, H), edge switches
    [H, H + E), aggregation switches [H + E, H + 2E) numbered pod * k/2 + a,
    core switches [H + 2E, ...) numbered a * k/2 + c; link ids are those of
    the fat-tree numbering (host links, edge-aggregation, aggregation-core).
    Returns (n_nodes, lu, lv) for residuals res[3H]."""
    half = k // 2
    H, E = k ** 3 // 4, k * k // 2
    lu = np.zeros(3 * H, np.int32)
    lv = np.zeros(3 * H, np.int32)
    for h in range(H):
        lu[h], lv[h] = h, H + h // half
    for e in range(E):
        p = e // half
        for a in range(half):
            lu[H + e * half + a], lv[H + e * half + a] = H + e, H + E + p * half + a
    for p in range(k):
        for a in range(half):
            for c in range(half):
                l = 2 * H + (p * half + a) * half + c
                lu[l], lv[l] = H + E + p * half + a, H + 2 * E + a * half + c
    return H + 2 * E + half * half, lu, lv


def utilities(q: Dict[str, np.ndarray], out: Dict[str, np.ndarray]):
    """U(i) per container and U(ij) per link of a scheduled request (Eqs. 1-2);
    `out` is what OracleDC.schedule returned."""
    rq = _Req(q)
    n, m = len(rq.a["pod"]), len(rq.a["src"])
    keep = {k: np.ascontiguousarray(out[k], np.int32) for k in ("host", "cpu", "mem", "bw", "path")}
    ps = np.ascontiguousarray(out["pod_score"], np.float64)
    res = _Result(int(out["status"]), int(out.get("n_decisions", 0)),
                  *(_p(keep[x], _i32p) for x in ("host", "cpu", "mem", "bw", "path")),
                  _p(ps, _f64p))
    uc = np.zeros(n, np.float64)
    ue = np.zeros(m, np.float64)
    lib().orc_utilities(C.byref(rq.s), C.byref(res), _p(uc, _f64p), _p(ue, _f64p))
    return uc, ue


def run_instance(inst, max_requests: Optional[int] = None) -> List[Dict[str, np.ndarray]]:
    """Runs the FCFS stream of an instance (schedules, and releases when the
    instance carries an operation list); returns one result per request."""
    dc = OracleDC.from_instance(inst)
    R = inst.reqs.n if max_requests is None else min(max_requests, inst.reqs.n)
    results: List[Optional[Dict[str, np.ndarray]]] = [None] * R
    ops = inst.ops if inst.ops is not None else [(0, r) for r in range(inst.reqs.n)]
    for kind, r in ops:
        if r >= R:
            if kind == 0:
                break
            continue
        if kind == 0:
            results[r] = dc.schedule(inst.reqs.request(r))
        elif results[r] is not None and results[r]["status"] == ACCEPTED:
            dc.release(inst.reqs.request(r), results[r])
    return results, dc


def _mat(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, np.int64))


def topsis(x, W) -> np.ndarray:
    x = _mat(x)
    F, Cn = x.shape
    out = np.zeros(F)
    w = np.ascontiguousarray(W, np.float64)
    lib().orc_topsis(F, Cn, _p(x, _i64p), _p(w, _f64p), _p(out, _f64p))
    return out


def ahp(x, W, rule=RATIO) -> np.ndarray:
    x = _mat(x)
    F, Cn = x.shape
    out = np.zeros(F)
    w = np.ascontiguousarray(W, np.float64)
    lib().orc_ahp(F, Cn, _p(x, _i64p), _p(w, _f64p), rule, _p(out, _f64p))
    return out


def ahp_literal(x, W, rule=RATIO) -> np.ndarray:
    x = _mat(x)
    F, Cn = x.shape
    out = np.zeros(F)
    w = np.ascontiguousarray(W, np.float64)
    lib().orc_ahp_literal(F, Cn, _p(x, _i64p), _p(w, _f64p), rule, _p(out, _f64p))
    return out


def ahp_weights(W, rule=RATIO) -> np.ndarray:
    w = np.ascontiguousarray(W, np.float64)
    out = np.zeros(len(w))
    lib().orc_ahp_weights(len(w), _p(w, _f64p), rule, _p(out, _f64p))
    return out

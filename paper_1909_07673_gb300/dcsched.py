"""ctypes binding of libdcsched.so (include/dcsched.h).

Argument marshalling only: every step of the scheduling path runs in the CUDA
library.  Importing this module without the built library raises; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdcsched.so")

TOPSIS, AHP, BF, WF = 0, 1, 2, 3
RATIO, DIFF = 0, 1
PENDING, ACCEPTED, REJECTED = 0, 1, 2
SCHED_SYNC, SCHED_ASYNC = 0, 1
PLAN_GRAPH, PLAN_RESET = 1, 2
FREE_CPU, FREE_MEM, CTR, PRE, LINK_RES = 0, 1, 2, 3, 4
E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_NOTFOUND, E_BUSY = -1, -2, -3, -4, -5, -6

_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f32p = C.POINTER(C.c_float)
_f64p = C.POINTER(C.c_double)


class DcError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s: %s (%d)" % (what, strerror(code), code))
        self.code = code


class _Config(C.Structure):
    _fields_ = [("k", C.c_int32), ("host_cpu", C.c_int32), ("host_mem", C.c_int32),
                ("link_mbps", C.c_int32), ("n_criteria", C.c_int32), ("method", C.c_int32),
                ("pair_rule", C.c_int32), ("weights", C.c_double * 6),
                ("pre_cpu", _i32p), ("pre_mem", _i32p), ("pre_link", _i32p)]


class _Request(C.Structure):
    _fields_ = [("n_containers", C.c_int32), ("n_edges", C.c_int32),
                ("cpu_min", _i32p), ("cpu_max", _i32p), ("mem_min", _i32p), ("mem_max", _i32p),
                ("pod", _i32p), ("src", _i32p), ("dst", _i32p), ("bw_min", _i32p),
                ("bw_max", _i32p)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_decisions", C.c_int32), ("host", _i32p),
                ("cpu", _i32p), ("mem", _i32p), ("bw", _i32p), ("path", _i32p),
                ("pod_score", _f64p), ("done_ns", C.c_int64)]


class _ServerStats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("requests", C.c_int64), ("decisions", C.c_int64),
                ("host_rankings", C.c_int64), ("peak_admitted_bytes", C.c_int64),
                ("wall_s", C.c_double)]


class _TuneEntry(C.Structure):
    _fields_ = [("k", C.c_int32), ("n_criteria", C.c_int32), ("method", C.c_int32),
                ("pair_rule", C.c_int32), ("block", C.c_int32), ("ncta", C.c_int32),
                ("block0", C.c_int32), ("ncta0", C.c_int32), ("trials", C.c_int32),
                ("kept", C.c_int32), ("ms", C.c_double), ("ms0", C.c_double)]


_lib = None


def lib():
    """Loads libdcsched.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdcsched.so not built: run __graft_entry__.build() "
                              "(or python -m paper_1909_07673_gb300.build)")
        L = C.CDLL(LIB_PATH)
        L.dc_strerror.restype = C.c_char_p
        L.dc_strerror.argtypes = [C.c_int]
        L.dc_create.argtypes = [C.POINTER(_Config), C.c_void_p, C.POINTER(C.c_void_p)]
        L.dc_destroy.argtypes = [C.c_void_p]
        L.dc_destroy.restype = None
        L.dc_submit_request.argtypes = [C.c_void_p, C.POINTER(_Request), _i64p]
        L.dc_submit_batch.argtypes = [C.c_void_p, C.c_int32, C.POINTER(_Request), _i64p]
        L.dc_io_stats.argtypes = [C.c_void_p, _i64p, _i64p]
        L.dc_release.argtypes = [C.c_void_p, C.c_int64]
        L.dc_schedule.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_int32]
        L.dc_query.argtypes = [C.c_void_p, C.c_int64, C.POINTER(_Result), C.c_int32]
        L.dc_query_state.argtypes = [C.c_void_p, C.c_int32, _i32p, C.c_int64]
        L.dc_rank_hosts.argtypes = [C.c_void_p, C.POINTER(_Request), C.c_int32, _i32p, _i32p,
                                    _f32p, _f64p, _i32p]
        L.dc_rank_hosts_static.argtypes = [C.c_void_p, C.POINTER(_Request), C.c_int32, _i32p,
                                           _i32p, _f32p, _f64p, _i32p]
        L.dc_reset.argtypes = [C.c_void_p]
        L.dc_server_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_int64, C.c_int32,
                                       C.POINTER(C.c_void_p)]
        L.dc_server_replay.argtypes = [C.c_void_p, C.c_int32, _f64p, _i32p, _i32p,
                                       C.POINTER(_Request), _i32p, _f64p, _i64p,
                                       C.POINTER(_ServerStats)]
        L.dc_server_set_timeout.argtypes = [C.c_void_p, C.c_double]
        L.dc_server_destroy.argtypes = [C.c_void_p]
        L.dc_server_destroy.restype = None
        L.dc_plan_create.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_int32,
                                     C.POINTER(C.c_void_p)]
        L.dc_plan_launch.argtypes = [C.c_void_p, C.c_void_p]
        L.dc_plan_collect.argtypes = [C.c_void_p]
        L.dc_plan_stats.argtypes = [C.c_void_p, _i64p, _i64p, _i32p, _i64p]
        L.dc_plan_diff_pairs.argtypes = [C.c_void_p, _i64p]
        L.dc_plan_destroy.argtypes = [C.c_void_p]
        L.dc_plan_destroy.restype = None
        L.dc_simulate.argtypes = [C.c_void_p, C.c_int32, _i32p, _i32p, _i32p]
        L.dc_utilities.argtypes = [C.c_void_p, C.c_int64, _f64p, _f64p]
        L.dc_utility_summary.argtypes = [C.c_void_p, _f64p, _i64p, _f64p, _i64p]
        L.dc_fragmentation.argtypes = [C.c_void_p, _i64p, _i64p, _f64p, _f64p]
        L.dc_graph_create.argtypes = [C.c_int32, C.c_int32, _i32p, _i32p, _i32p, C.c_void_p,
                                      C.POINTER(C.c_void_p)]
        L.dc_graph_destroy.argtypes = [C.c_void_p]
        L.dc_graph_destroy.restype = None
        L.dc_graph_set_residual.argtypes = [C.c_void_p, _i32p]
        L.dc_graph_widest_paths.argtypes = [C.c_void_p, C.c_int32, _i32p, _i32p, C.c_int32,
                                            _i32p, _i32p, _i32p]
        L.dc_set_launch.argtypes = [C.c_int32] * 6
        L.dc_get_launch.argtypes = [C.c_void_p, _i32p, _i32p, _i64p]
        L.dc_autotune.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.c_int32,
                                  C.POINTER(_TuneEntry), C.c_int32, _i32p]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().dc_strerror(code).decode()


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise DcError(rc, what)
    return rc


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _stream_handle(stream) -> Optional[int]:
    """Accepts None, an int handle or an object with .cuda_stream (torch)."""
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


class _Req:
    def __init__(self, q: Dict[str, np.ndarray]):
        self.a = {k: np.ascontiguousarray(q[k], np.int32) for k in (
            "cpu_min", "cpu_max", "mem_min", "mem_max", "pod", "src", "dst", "bw_min", "bw_max")}
        a = self.a
        self.s = _Request(len(a["pod"]), len(a["src"]), *(_p(a[n], _i32p) for n in (
            "cpu_min", "cpu_max", "mem_min", "mem_max", "pod", "src", "dst", "bw_min", "bw_max")))
        self.n_pods = int(a["pod"].max()) + 1 if len(a["pod"]) else 0


class DataCenter:
    """One resident data center (dc_t)."""

    def __init__(self, k, host_cpu, host_mem, link_mbps, n_criteria, method, pair_rule, weights,
                 pre_cpu=None, pre_mem=None, pre_link=None, stream=None):
        w = (C.c_double * 6)(*([float(x) for x in weights] + [0.0] * (6 - len(weights))))
        keep = [None if a is None else np.ascontiguousarray(a, np.int32)
                for a in (pre_cpu, pre_mem, pre_link)]
        cfg = _Config(k, host_cpu, host_mem, link_mbps, n_criteria, method, pair_rule, w,
                      *(None if a is None else _p(a, _i32p) for a in keep))
        h = C.c_void_p()
        _check(lib().dc_create(C.byref(cfg), _stream_handle(stream), C.byref(h)), "dc_create")
        self.h = h
        self.k = k
        self.H = k ** 3 // 4
        self.n_criteria = n_criteria
        self._reqs: List[_Req] = []

    @classmethod
    def from_instance(cls, inst, stream=None) -> "DataCenter":
        return cls(inst.k, inst.host_cpu, inst.host_mem, inst.link_mbps, inst.n_criteria,
                   inst.method, inst.pair_rule, inst.weights, inst.pre_cpu, inst.pre_mem,
                   inst.pre_link, stream=stream)

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def submit(self, q: Dict[str, np.ndarray]) -> int:
        r = _Req(q)
        rid = C.c_int64()
        _check(lib().dc_submit_request(self.h, C.byref(r.s), C.byref(rid)), "dc_submit_request")
        self._reqs.append(r)
        return rid.value

    def release(self, req_id: int) -> None:
        _check(lib().dc_release(self.h, req_id), "dc_release")

    def query(self, req_id: int, wait: bool = True) -> Dict[str, np.ndarray]:
        r = self._reqs[req_id]
        n, m, P = len(r.a["pod"]), len(r.a["src"]), r.n_pods
        out = {"host": np.zeros(n, np.int32), "cpu": np.zeros(n, np.int32),
               "mem": np.zeros(n, np.int32), "bw": np.zeros(m, np.int32),
               "path": np.zeros(6 * m, np.int32), "pod_score": np.zeros(P, np.float64)}
        res = _Result(0, 0, *(_p(out[x], _i32p) for x in ("host", "cpu", "mem", "bw", "path")),
                      _p(out["pod_score"], _f64p), 0)
        _check(lib().dc_query(self.h, req_id, C.byref(res), 1 if wait else 0), "dc_query")
        out["status"] = int(res.status)
        out["n_decisions"] = int(res.n_decisions)
        out["done_ns"] = int(res.done_ns)
        return out

    def status(self, req_id: int, wait: bool = True):
        """(status, n_decisions, done_ns) without copying the placement."""
        res = _Result(0, 0, None, None, None, None, None, None, 0)
        _check(lib().dc_query(self.h, req_id, C.byref(res), 1 if wait else 0), "dc_query")
        return int(res.status), int(res.n_decisions), int(res.done_ns)

    def submit_batch(self, batch) -> int:
        """Submits every request of a workloads.RequestBatch in order with one
        call; returns the id of the first."""
        reqs = [_Req(batch.request(r)) for r in range(batch.n)]
        arr = (_Request * len(reqs))(*[r.s for r in reqs])
        ids = np.zeros(max(1, len(reqs)), np.int64)
        _check(lib().dc_submit_batch(self.h, len(reqs), arr, _p(ids, _i64p)), "dc_submit_batch")
        self._reqs.extend(reqs)
        return int(ids[0])

    def simulate(self, n_steps: int, submit_step, duration) -> np.ndarray:
        """Discrete-event simulation of the queued requests (dc_simulate);
        returns each one's start step (-1: never started)."""
        sub = np.ascontiguousarray(submit_step, np.int32)
        dur = np.ascontiguousarray(duration, np.int32)
        start = np.zeros(max(1, len(sub)), np.int32)
        _check(lib().dc_simulate(self.h, int(n_steps), _p(sub, _i32p), _p(dur, _i32p),
                                 _p(start, _i32p)), "dc_simulate")
        return start[:len(sub)]

    def utilities(self, req_id: int):
        """(U(i) per container, U(ij) per link) of a scheduled request
        (Eqs. 1-2, dc_utilities)."""
        r = self._reqs[req_id]
        uc = np.zeros(len(r.a["pod"]), np.float64)
        ue = np.zeros(len(r.a["src"]), np.float64)
        _check(lib().dc_utilities(self.h, req_id, _p(uc, _f64p), _p(ue, _f64p)), "dc_utilities")
        return uc, ue

    def utility_summary(self) -> Dict[str, float]:
        """Sums of U(i) / U(ij) over the accepted requests scheduled so far and
        the numbers of containers / links (dc_utility_summary)."""
        a, b = C.c_double(), C.c_double()
        n, m = C.c_int64(), C.c_int64()
        _check(lib().dc_utility_summary(self.h, C.byref(a), C.byref(n), C.byref(b), C.byref(m)),
               "dc_utility_summary")
        return {"sum_u_container": a.value, "n_containers": n.value, "sum_u_link": b.value,
                "n_links": m.value}

    def fragmentation(self):
        """(active servers, active links, F(N^s), F(E^s)) of the current state
        (dc_fragmentation)."""
        a, b = C.c_int64(), C.c_int64()
        fs, fl = C.c_double(), C.c_double()
        _check(lib().dc_fragmentation(self.h, C.byref(a), C.byref(b), C.byref(fs), C.byref(fl)),
               "dc_fragmentation")
        return a.value, b.value, fs.value, fl.value

    def io_stats(self):
        a, b = C.c_int64(), C.c_int64()
        _check(lib().dc_io_stats(self.h, C.byref(a), C.byref(b)), "dc_io_stats")
        return a.value, b.value

    def state(self, field: int) -> np.ndarray:
        n = 3 * self.H if field == LINK_RES else self.H
        a = np.zeros(n, np.int32)
        _check(lib().dc_query_state(self.h, field, _p(a, _i32p), n), "dc_query_state")
        return a

    def rank_hosts(self, q: Dict[str, np.ndarray], pod: int, host_of: np.ndarray):
        r = _Req(q)
        ho = np.ascontiguousarray(host_of, np.int32)
        feas = np.zeros(self.H, np.int32)
        s32 = np.zeros(self.H, np.float32)
        s64 = np.zeros(self.H, np.float64)
        crit = np.zeros(self.H * self.n_criteria, np.int32)
        nv = _check(lib().dc_rank_hosts(self.h, C.byref(r.s), pod, _p(ho, _i32p), _p(feas, _i32p),
                                        _p(s32, _f32p), _p(s64, _f64p), _p(crit, _i32p)),
                    "dc_rank_hosts")
        return feas.astype(bool), s32, s64, crit.reshape(self.H, self.n_criteria), nv

    def rank_hosts_static(self, q: Dict[str, np.ndarray], pod: int, host_of: np.ndarray):
        """rank_hosts through the allocation-free entry point (device
        temporaries in the library's static scratch array)."""
        r = _Req(q)
        ho = np.ascontiguousarray(host_of, np.int32)
        feas = np.zeros(self.H, np.int32)
        s32 = np.zeros(self.H, np.float32)
        s64 = np.zeros(self.H, np.float64)
        crit = np.zeros(self.H * self.n_criteria, np.int32)
        nv = _check(lib().dc_rank_hosts_static(self.h, C.byref(r.s), pod, _p(ho, _i32p),
                                               _p(feas, _i32p), _p(s32, _f32p), _p(s64, _f64p),
                                               _p(crit, _i32p)), "dc_rank_hosts_static")
        return feas.astype(bool), s32, s64, crit.reshape(self.H, self.n_criteria), nv

    def reset(self) -> None:
        _check(lib().dc_reset(self.h), "dc_reset")
        self._reqs = []


def _handles(dcs: Sequence[DataCenter]):
    arr = (C.c_void_p * len(dcs))(*[d.h.value for d in dcs])
    return arr


def schedule(dcs: Sequence[DataCenter], flags: int = SCHED_SYNC) -> None:
    _check(lib().dc_schedule(_handles(dcs), len(dcs), flags), "dc_schedule")


class Plan:
    """A prepared batched launch (dc_plan)."""

    def __init__(self, dcs: Sequence[DataCenter], flags: int = 0):
        self.dcs = list(dcs)
        h = C.c_void_p()
        _check(lib().dc_plan_create(_handles(self.dcs), len(self.dcs), flags, C.byref(h)),
               "dc_plan_create")
        self.h = h

    def launch(self, stream=None) -> None:
        _check(lib().dc_plan_launch(self.h, _stream_handle(stream)), "dc_plan_launch")

    def collect(self) -> None:
        _check(lib().dc_plan_collect(self.h), "dc_plan_collect")

    def stats(self):
        """(decisions, host rankings, kernels per launch, start clock ns)"""
        d, hr, kc, t0 = C.c_int64(), C.c_int64(), C.c_int32(), C.c_int64()
        _check(lib().dc_plan_stats(self.h, C.byref(d), C.byref(hr), C.byref(kc), C.byref(t0)),
               "dc_plan_stats")
        return d.value, hr.value, kc.value, t0.value

    def diff_pairs(self) -> int:
        """AHP DIFF pair evaluations (2 sum_v D_v^2 over the decisions) of the
        last collected launch (dc_plan_diff_pairs)."""
        n = C.c_int64()
        _check(lib().dc_plan_diff_pairs(self.h, C.byref(n)), "dc_plan_diff_pairs")
        return n.value

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dc_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Server:
    """Continuous-batching serving loop over resident data centers (dc_server)."""

    def __init__(self, dcs: Sequence[DataCenter], admit_bytes: int = 1 << 30,
                 max_requests_per_launch: int = 0, stall_s: Optional[float] = None):
        self.dcs = list(dcs)
        h = C.c_void_p()
        _check(lib().dc_server_create(_handles(self.dcs), len(self.dcs), admit_bytes,
                                      max_requests_per_launch, C.byref(h)), "dc_server_create")
        self.h = h
        if stall_s is not None:
            _check(lib().dc_server_set_timeout(h, stall_s), "dc_server_set_timeout")

    def replay(self, t, inst, kind, reqs, release_of):
        """Replays timed events (see dc_server_replay); reqs[i] is a request
        dict for kind-0 events (None otherwise).  Returns (latency_s,
        req_id, stats dict).  The request ids are registered with the data
        centers' bindings so that DataCenter.query works afterwards."""
        n = len(t)
        t = np.ascontiguousarray(t, np.float64)
        inst = np.ascontiguousarray(inst, np.int32)
        kind = np.ascontiguousarray(kind, np.int32)
        rel = np.ascontiguousarray(release_of, np.int32)
        keep = [(_Req(q) if q is not None else None) for q in reqs]
        arr = (_Request * max(1, n))(*[(r.s if r is not None else _Request()) for r in keep])
        lat = np.zeros(n, np.float64)
        rid = np.zeros(n, np.int64)
        st = _ServerStats()
        _check(lib().dc_server_replay(self.h, n, _p(t, _f64p), _p(inst, _i32p), _p(kind, _i32p),
                                      arr, _p(rel, _i32p), _p(lat, _f64p), _p(rid, _i64p),
                                      C.byref(st)), "dc_server_replay")
        for e in range(n):
            if kind[e] == 0:
                d = self.dcs[inst[e]]
                assert rid[e] == len(d._reqs)
                d._reqs.append(keep[e])
        stats = {f: getattr(st, f) for f, _ in _ServerStats._fields_}
        return lat, rid, stats

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.dc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Graph:
    """A general data-center graph with per-link residual bandwidth on the
    device (dc_graph); widest_paths runs the widest-shortest-path search for
    many (source, destination) pairs in one kernel."""

    def __init__(self, n_nodes: int, link_u, link_v, residual, stream=None):
        lu = np.ascontiguousarray(link_u, np.int32)
        lv = np.ascontiguousarray(link_v, np.int32)
        res = np.ascontiguousarray(residual, np.int32)
        h = C.c_void_p()
        _check(lib().dc_graph_create(int(n_nodes), len(lu), _p(lu, _i32p), _p(lv, _i32p),
                                     _p(res, _i32p), _stream_handle(stream), C.byref(h)),
               "dc_graph_create")
        self.h = h
        self.V, self.L = int(n_nodes), len(lu)

    def set_residual(self, residual) -> None:
        res = np.ascontiguousarray(residual, np.int32)
        _check(lib().dc_graph_set_residual(self.h, _p(res, _i32p)), "dc_graph_set_residual")

    def widest_paths(self, src, dst, max_hops: int = 16):
        """(hops, bottleneck, links[n, max_hops]) per pair."""
        s = np.ascontiguousarray(src, np.int32)
        d = np.ascontiguousarray(dst, np.int32)
        n = len(s)
        hops = np.zeros(n, np.int32)
        bott = np.zeros(n, np.int32)
        links = np.full(max(1, n * max_hops), -1, np.int32)
        _check(lib().dc_graph_widest_paths(self.h, n, _p(s, _i32p), _p(d, _i32p), max_hops,
                                           _p(hops, _i32p), _p(bott, _i32p), _p(links, _i32p)),
               "dc_graph_widest_paths")
        return hops, bott, links[:n * max_hops].reshape(n, max_hops)

    def close(self) -> None:
        if getattr(self, "h", None) and _lib is not None:
            _lib.dc_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


def set_launch(k: int, n_criteria: int, method: int, pair_rule: int, block: int,
               ncta: int = 1) -> None:
    """Records the scheduling-kernel shape (threads per block, blocks per
    data center) for data centers of this kind (dc_set_launch); block 0
    removes the entry."""
    _check(lib().dc_set_launch(k, n_criteria, method, pair_rule, block, ncta), "dc_set_launch")


def autotune(dcs: Sequence["DataCenter"], max_ops: int = 0) -> List[Dict[str, float]]:
    """Chooses the launch shape of every kind of data center among dcs for
    the batched launch of their queued operations (dc_autotune; only the
    first max_ops operations of each, 0 = all) and records it.  Returns one
    dict per kind."""
    out = (_TuneEntry * 64)()
    n = C.c_int32()
    _check(lib().dc_autotune(_handles(list(dcs)), len(dcs), max_ops, out, 64, C.byref(n)),
           "dc_autotune")
    return [{f: getattr(out[i], f) for f, _ in _TuneEntry._fields_}
            for i in range(min(n.value, 64))]


def get_launch(dc: "DataCenter"):
    """(block, blocks per data center, dynamic shared memory bytes) a plan
    would use for dc."""
    b, n, sm = C.c_int32(), C.c_int32(), C.c_int64()
    _check(lib().dc_get_launch(dc.h, C.byref(b), C.byref(n), C.byref(sm)), "dc_get_launch")
    return b.value, n.value, sm.value


def load_instance(inst, stream=None, max_requests: Optional[int] = None) -> DataCenter:
    """Creates a DataCenter for a workloads.Instance and submits its FCFS
    stream of operations (schedules and releases)."""
    dc = DataCenter.from_instance(inst, stream=stream)
    R = inst.reqs.n if max_requests is None else min(max_requests, inst.reqs.n)
    if inst.ops is None:
        dc.submit_batch(inst.reqs if R == inst.reqs.n else inst.reqs.subset(range(R)))
        return dc
    ops = inst.ops
    for kind, r in ops:
        if r >= R:
            if kind == 0:
                break
            continue
        if kind == 0:
            dc.submit(inst.reqs.request(r))
        else:
            dc.release(r)
    return dc

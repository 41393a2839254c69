"""Helpers comparing the CUDA path (through the C-ABI binding) with the
FP64 oracle on the same seeded inputs."""
import numpy as np

import oracle as O

KEYS = ("host", "cpu", "mem", "bw", "path", "pod_score")


def assert_same_result(got, exp, where):
    assert got["status"] == exp["status"], (where, "status", got["status"], exp["status"])
    assert got["n_decisions"] == exp["n_decisions"], (where, "n_decisions")
    for key in KEYS:
        g, e = got[key], exp[key]
        if not np.array_equal(g, e):
            bad = np.nonzero(g != e)[0][:8]
            raise AssertionError("%s: %s differs at %s: gpu %s oracle %s" % (
                where, key, bad.tolist(), g[bad].tolist(), e[bad].tolist()))


def assert_same_state(dc, odc, where):
    for f in (O.FREE_CPU, O.FREE_MEM, O.CTR, O.LINK_RES):
        g, e = dc.state(f), odc.state(f)
        if not np.array_equal(g, e):
            bad = np.nonzero(g != e)[0][:8]
            raise AssertionError("%s: state field %d differs at %s: gpu %s oracle %s" % (
                where, f, bad.tolist(), g[bad].tolist(), e[bad].tolist()))


def check_instance(dc, inst, max_requests=None, where=""):
    """dc has been scheduled; compares every request and the final state."""
    ref, odc = O.run_instance(inst, max_requests=max_requests)
    R = len(ref)
    for r in range(R):
        if ref[r] is None:
            continue
        assert_same_result(dc.query(r), ref[r], "%s req %d" % (where, r))
    assert_same_state(dc, odc, where)
    return ref


def gpu_results(dc, n):
    """Results of requests 0..n-1 of a scheduled data center, and its final
    integer state, read through the C-ABI (on the calling thread)."""
    res = [dc.query(r) for r in range(n)]
    state = {f: dc.state(f) for f in (O.FREE_CPU, O.FREE_MEM, O.CTR, O.LINK_RES)}
    return res, state


def compare_chain(inst, got, state, where, max_requests=None):
    """Runs the oracle over the instance's FCFS stream and compares every
    request and the final state with what the GPU produced; returns an error
    message or None.  Thread-safe (the oracle's C calls release the
    interpreter lock, so a pool of threads runs data centers in parallel)."""
    try:
        ref, odc = O.run_instance(inst, max_requests=max_requests)
        for r in range(len(ref)):
            if ref[r] is not None:
                assert_same_result(got[r], ref[r], "%s req %d" % (where, r))
        for f, g in state.items():
            e = odc.state(f)
            if not np.array_equal(g, e):
                bad = np.nonzero(g != e)[0][:8]
                raise AssertionError("%s: state field %d differs at %s" % (where, f, bad.tolist()))
    except AssertionError as e:
        return str(e)
    return None


def compare_chains(jobs, threads=None):
    """jobs: (instance, gpu results, gpu state, label, max_requests); runs
    compare_chain over a thread pool; returns the list of error messages."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    n = threads or max(1, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=n) as ex:
        errs = list(ex.map(lambda j: compare_chain(*j), jobs))
    return [e for e in errs if e]

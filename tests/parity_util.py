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

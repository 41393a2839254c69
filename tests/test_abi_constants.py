"""The Python binding's constants equal the enum values declared in
include/dcsched.h (methods, pair rules, statuses, flags, state fields, error
codes), so that no code crosses the boundary with another meaning.  CPU
only (reads the header as text)."""
import os
import re

from paper_1909_07673_gb300 import dcsched as ds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_enums():
    txt = open(os.path.join(ROOT, "include", "dcsched.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", txt, flags=re.S):
        for name, val in re.findall(r"\b(DC_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            vals[name] = int(val)
    return vals


def test_binding_constants_match_header():
    h = _header_enums()
    pairs = {
        "DC_TOPSIS": ds.TOPSIS, "DC_AHP": ds.AHP, "DC_BF": ds.BF, "DC_WF": ds.WF,
        "DC_PAIR_RATIO": ds.RATIO, "DC_PAIR_DIFF": ds.DIFF,
        "DC_PENDING": ds.PENDING, "DC_ACCEPTED": ds.ACCEPTED, "DC_REJECTED": ds.REJECTED,
        "DC_SCHED_SYNC": ds.SCHED_SYNC, "DC_SCHED_ASYNC": ds.SCHED_ASYNC,
        "DC_PLAN_GRAPH": ds.PLAN_GRAPH, "DC_PLAN_RESET": ds.PLAN_RESET,
        "DC_FIELD_FREE_CPU": ds.FREE_CPU, "DC_FIELD_FREE_MEM": ds.FREE_MEM,
        "DC_FIELD_CTR": ds.CTR, "DC_FIELD_PRE": ds.PRE, "DC_FIELD_LINK_RES": ds.LINK_RES,
        "DC_E_INVAL": ds.E_INVAL, "DC_E_NOMEM": ds.E_NOMEM, "DC_E_CUDA": ds.E_CUDA,
        "DC_E_TIMEOUT": ds.E_TIMEOUT, "DC_E_NOTFOUND": ds.E_NOTFOUND, "DC_E_BUSY": ds.E_BUSY,
    }
    for name, value in pairs.items():
        assert name in h, name
        assert h[name] == value, (name, h[name], value)


def test_error_codes_are_distinct_and_negative():
    h = _header_enums()
    errs = {k: v for k, v in h.items() if k.startswith("DC_E_")}
    assert h["DC_OK"] == 0
    assert errs and all(v < 0 for v in errs.values())
    assert len(set(errs.values())) == len(errs)

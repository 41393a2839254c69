"""The C-ABI library builds, loads and exports every entry point declared in
include/dcsched.h (no compute call: runs without a GPU)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "dcsched.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dc_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dc_create", "dc_destroy", "dc_submit_request", "dc_release", "dc_schedule",
              "dc_query", "dc_query_state", "dc_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1909_07673_gb300 import build

    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(dc_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    h = ctypes.CDLL(lib)
    for n in _declared():
        assert getattr(h, n) is not None
    h.dc_strerror.restype = ctypes.c_char_p
    assert h.dc_strerror(-1) == b"invalid argument or request"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1909_07673_gb300 import dcsched

    monkeypatch.setattr(dcsched, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(dcsched, "_lib", None)
    try:
        dcsched.lib()
    except ImportError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("no error without the library")

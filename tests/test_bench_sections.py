"""bench.py's optional sections: a failing section is reported in its own key
and does not cost the main JSON line (no GPU needed)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_failing_section_reported_in_its_key(capsys):
    def boom(n):
        raise RuntimeError("section broke at %d" % n)

    out = bench.optional_section("demo", boom, 7)
    assert out == {"error": "RuntimeError: section broke at 7"}
    assert "section demo failed" in capsys.readouterr().err


def test_passing_section_returns_its_value():
    assert bench.optional_section("demo", lambda a, b: {"sum": a + b}, 2, 3) == {"sum": 5}


def test_oracle_sample_runs_whole_chains():
    """The CPU baseline and the reference arm time whole FCFS chains (every
    request of each data center taken), and count host rankings as the
    oracle's decisions times the data center's hosts."""
    import oracle as O
    from paper_1909_07673_gb300 import workloads as W

    wl = W.batched(n_instances=4, n_requests=3, ks=(4, 8), size_hi=12)
    hr, wall, desc, reqs, threads = bench.oracle_sample(wl, seconds=60.0, threads=2)
    assert reqs == 4 * 3 and threads == 2 and wall > 0
    exp = 0
    for inst in wl.instances:
        ref, _ = O.run_instance(inst)
        exp += sum(r["n_decisions"] for r in ref) * inst.hosts
    assert hr == exp
    assert "whole 3-request chains of 4 data centers" in desc

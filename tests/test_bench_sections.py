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

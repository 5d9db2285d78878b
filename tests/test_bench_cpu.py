"""Host arithmetic of bench.py's roofline on CPU: the per-phase and overall
HBM fractions from a hand-made profile, whose numbers are checked by hand."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_phase_roofline_by_hand():
    sys.path.insert(0, ROOT)
    import bench
    prof = {
        ("move", "sweep"): {"launches": 4, "ms": 2.0, "bytes": 8e9},
        ("move", "block"): {"launches": 1, "ms": 2.0, "bytes": 2e9},
        ("refine", "sweep"): {"launches": 2, "ms": 1.0, "bytes": 1e9},
        ("aggregate", "warp"): {"launches": 1, "ms": 5.0, "bytes": 1e9},
    }
    by, over = bench.phase_roofline(prof, 1000.0, 20.0)
    # move: 10 GB in 4 ms = 2500 GB/s; refine: 1 GB in 1 ms; aggregate: 1 GB in 5 ms
    assert by["move"]["launches"] == 5
    assert by["move"]["achieved"] == pytest.approx(2500.0)
    assert by["move"]["frac"] == pytest.approx(2.5)
    assert by["refine"]["achieved"] == pytest.approx(1000.0)
    assert by["aggregate"]["achieved"] == pytest.approx(200.0)
    # 12 GB over the 10 profiled ms and over the 20 ms step
    assert over["bytes"] == pytest.approx(12e9)
    assert over["achieved_profiled"] == pytest.approx(1200.0)
    assert over["frac_profiled"] == pytest.approx(1.2)
    assert over["achieved_step"] == pytest.approx(600.0)
    assert over["frac_step"] == pytest.approx(0.6)


def test_phase_roofline_empty_profile():
    sys.path.insert(0, ROOT)
    import bench
    by, over = bench.phase_roofline({}, 1000.0, 5.0)
    assert by == {}
    assert over["achieved_step"] == 0.0 and over["achieved_profiled"] == 0.0

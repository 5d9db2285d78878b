"""Host side of bench.py on CPU: the roofline arithmetic from a hand-made
profile (numbers checked by hand) and the reference arm's JSON line."""
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


def _bench(args, env_extra=None):
    import json
    import subprocess
    env = dict(os.environ, **(env_extra or {}))
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line():
    """The reference arm (the oracle on host cores) prints one JSON line with
    the contract's keys, the same metric and unit as the GPU arm, and an e2e
    that moves no bytes."""
    (line,) = _bench(["--impl", "reference", "--workload", "road", "--steps", "2", "--warmup", "1",
                      "--ref-side", "60"])
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "edges/s"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "edges/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert 0.5 < line["config"]["modularity"] < 1.0


def test_reference_arm_rmat_sample():
    """The default workload's reference arm runs the oracle on a bounded
    sample of the same R-MAT recipe and names it."""
    (line,) = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-scale", "10"])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"].startswith("R-MAT scale 10, edge factor 56")
    assert "bounded sample of the scale-25 workload" in line["config"]["workload"]
    assert 0.0 < line["config"]["modularity"] < 0.5


def test_reference_arm_other_ranks_silent():
    """Under torchrun only rank 0 runs the oracle; the others exit 0 quietly."""
    assert _bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-side", "60"],
                  {"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_optional_leg_reports_a_failure_in_its_place(capsys):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.optional_leg(lambda a, b: a + b, 2, 3) == 5

    def broken():
        raise ValueError("no such graph")
    assert bench.optional_leg(broken) == {"error": "ValueError: no such graph"}
    assert "no such graph" in capsys.readouterr().err


def test_traffic_lookup(tmp_path, monkeypatch):
    """The DRAM traffic of the committed ncu summary is reported only for the
    same kernel sources and workload; a capture of a smaller case of the same
    recipe is carried beside a workload too large to capture, not as its
    traffic."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    f = tmp_path / "traffic.json"
    h = bench.kernel_source_hash()
    cap = {"move/sweep": {"dram_bytes_per_launch": 7.0e9, "algorithmic_bytes_per_launch": 3.5e9, "ratio": 2.0}}
    f.write_text(json.dumps({"source_hash": h, "captures": [
        {"workload": "road A", "classes": {"move/sweep": {"dram_bytes_per_launch": 4.0e9}}},
        {"workload": "R-MAT small", "stands_for": "R-MAT large", "classes": cap}]}))
    monkeypatch.setattr(bench, "TRAFFIC", str(f))
    assert bench.traffic_for("move/sweep", "road A") == (4.0e9, None)
    exact, sample = bench.traffic_for("move/sweep", "R-MAT large")
    assert exact is None and sample["workload"] == "R-MAT small" and sample["ratio"] == 2.0
    assert bench.traffic_for("refine/sweep", "road A") == (None, None)
    assert bench.traffic_for("move/sweep", "another workload") == (None, None)
    # other kernel sources: nothing
    f.write_text(json.dumps({"source_hash": "0" * 16, "captures": [
        {"workload": "road A", "classes": {"move/sweep": {"dram_bytes_per_launch": 4.0e9}}}]}))
    assert bench.traffic_for("move/sweep", "road A") == (None, None)

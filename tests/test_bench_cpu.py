"""The reference arm of bench.py (the FP64 oracle on the host cores) prints one JSON line with
the keys of the benchmark contract; no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ref-poses", "64",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "queries/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] >= 3 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["poses_per_step"] == 64


def test_clock_summary_keeps_the_marked_window():
    """Samples before the first mark (an idle GPU) and after the last are left out; a throttle
    reason seen inside the window is reported."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler()
    row = "0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, {th}, Not Active"
    c.lines = [(0.0, row.format(sm=345, th="Not Active")),          # idle, before the window
               (1.0, row.format(sm=2070, th="Not Active")),
               (1.2, row.format(sm=2055, th="Active")),
               (9.0, row.format(sm=345, th="Not Active"))]         # after the window
    c.marks = [0.95, 1.25]
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == (2070 + 2055) / 2 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_thermal_slowdown"]
    c.marks = [5.0, 5.05]
    assert c.summary()["reasons"] == ["unsampled"]

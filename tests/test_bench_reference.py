"""The benchmark's reference arm (the CPU oracle, no GPU): one JSON line with the
contract's keys, on a small workload so that it runs in seconds."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "unigrid64", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_net_fraction_bounds_the_raw_one_from_above():
    """The roofline fraction net of the event-pair floor: the raw fraction scaled by
    duration / (duration - floor), None when the floor is unknown or not below the
    duration."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.net_frac(0.5, 0.010, 5.0) == 0.5 * 10.0 / 5.0
    assert bench.net_frac(0.5, 0.010, 0.0) == 0.5
    assert bench.net_frac(0.5, 0.010, None) is None
    assert bench.net_frac(0.5, 0.004, 5.0) is None
    assert bench.net_frac(0.5, None, 1.0) is None

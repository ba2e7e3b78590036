"""Host-side parts of bench.py: the reference arm (the oracle timed on this
host's cores) prints one JSON line in the benchmark's format, and the error
and drift summaries are computed as stated."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"] and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("kerr_camera_a0.9_1024x1024")


def test_drift_and_error_summaries():
    sys.path.insert(0, ROOT)
    import torch

    import bench

    inv0 = np.array([[1.0, 2.0, 0.5], [3.0, -3.0, 0.1], [0.0, 5.0, 7.0], [-1.0, -1.0, -1.0]])
    inv1 = inv0.copy()
    inv1[0, 1] += 2e-6 * 2.0  # relative 2e-6
    inv1[2, 0] = 1e-7         # |inv0| < 1: absolute 1e-7
    inv1[3, 2] = np.nan
    d = bench.drift_stats(inv0, inv1)
    assert abs(d["E"]["max"] - 2e-6) < 1e-12 and abs(d["E"]["frac_le_1e-6"] - 2 / 3) < 1e-12
    assert abs(d["Q"]["max"] - 1e-7) < 1e-15 and d["Lz"]["max"] == 0.0
    assert d["norm"]["nonfinite"] == 1
    dth = torch.tensor([0.0, 1e-9, 1e-3, 2.0], dtype=torch.float64)
    e = bench.err_stats(torch, dth, dth)
    assert e["rays"] == 4 and e["theta"]["max"] == 2.0 and e["theta"]["above_1e-6"] == 2

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


def _free_port() -> int:
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ranks_worker(rank, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": "2",
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench

    r = bench.Ranks.from_env()
    r.barrier()
    q.put((rank, r.max(1.5 + rank)))
    r.close()


def test_ranks_barrier_and_max_over_gloo():
    """The bench's multi-rank plumbing (one process per GPU under torchrun):
    two gloo ranks on the host agree on the maximum of their timings."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_ranks_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_reference_arm_under_torchrun_prints_once():
    """--impl reference launched the way the driver launches N > 1: rank 0
    prints one JSON line, the other rank exits 0 without work."""
    port = _free_port()
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2


def test_self_convergence_ratio_and_drift_summary():
    """bench.q_ratio is the paper's Q = |y_h - y_h/2| / |y_h/2 - y_h/4| per ray
    (largest component difference), leaving out non-finite and vanishing
    differences; bench.drift_summary reports |inv1 - inv0| without the
    non-finite rays."""
    sys.path.insert(0, ROOT)
    import torch

    import bench

    base = np.zeros((8, 4))
    f1, f2, f3 = base.copy(), base.copy(), base.copy()
    f1[1] = [16e-6, 8e-6, 1.0, np.nan]
    f2[1] = [1e-6, 1e-6, 1.0, 0.0]
    f3[1] = [0.0, 0.0, 1.0, 0.0]
    q = bench.q_ratio([f1, f2, f3])
    assert q["rays"] == 2 and q["of"] == 4
    assert abs(q["median"] - 11.0) < 1e-9 and q["frac_13_19"] == 0.5  # Q = 15 and 7

    class FakeMb:
        FATE_NONFINITE = 4
        FATE_MASK, FATE_DRIFTED = 0x7F, 0x80

    # a flagged CAPPED ray (0x83) counts as CAPPED: only the NONFINITE one is left out
    r = {"fate": torch.tensor([3, 0x83, 4, 2]),
         "inv0": torch.ones((4, 4), dtype=torch.float64),
         "inv1": torch.ones((4, 4), dtype=torch.float64)}
    r["inv1"][2] += torch.tensor([1e-9, 3e-9, 1e3, 2e-9], dtype=torch.float64)
    d = bench.drift_summary(FakeMb, torch, r)
    assert d["nonfinite"] == 1 and abs(d["Q"]["median"] - 2e-9) < 1e-15 and d["E"]["median"] == 0.0


def test_fate_counts_split_the_validity_flag():
    """bench.fate_counts counts terminations by fate & FATE_MASK and the
    flagged (FATE_DRIFTED) escaped and capped rays separately."""
    sys.path.insert(0, ROOT)
    import torch

    import bench

    class FakeMb:
        FATE_MASK, FATE_DRIFTED = 0x7F, 0x80

    f = torch.tensor([1, 2, 0x82, 0x82, 3, 0x83, 4, 2], dtype=torch.uint8)
    c = bench.fate_counts(FakeMb, f)
    assert c["captured"] == 1 and c["escaped"] == 4 and c["escaped_drifted"] == 2
    assert c["capped"] == 2 and c["capped_drifted"] == 1 and c["nonfinite"] == 1
    assert abs(c["drifted_fraction"] - 3 / 8) < 1e-12

"""Benchmark: RK4 geodesic steps/s on the Kerr a = 0.9 backward camera.

Workload (one bench step): render the 1024 x 1024 backward null-ray camera of
a Kerr black hole with a = 0.9M, observer at 1000M, inclination 80 deg,
impact parameters in +-25M, RK4 step 0.05 r, cap 2x10^4 steps, stop at
1.01 r_+ or r > 1100M, FP64.  The metric counts every RK4 step every ray took.
Beside it the same render in FP32_MIXED, the end-to-end number through the
host-buffer C-ABI entry point, the roofline of the trace kernel, and the CPU
oracle timed on this host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank renders its own image (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RK4 geodesic steps/s at stated error vs FP64 oracle; p50/p99 request latency"
UNIT = "steps/s"
WORKLOAD = "kerr_camera_a0.9_1024x1024_incl80_fov25_h0.05r_cap2e4"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
KERNEL_SOURCES = ["geodesic.cuh", "camera.cuh", "trace.cu"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1803_08320_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# algorithmic flops per RK4 step, counted from the kernel source expressions
# (FMA = 2, add/mul = 1); divisions and sincos are listed separately (4 each)
FLOPS_PER_STEP = {"kerr": 4 * 131 + 96, "schw": 4 * 42 + 96}
DIV_PER_STEP, SINCOS_PER_STEP = 4, 4


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"malbec_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append({"sm": float(parts[1]), "max": float(parts[2]), "power": float(parts[3]),
                             "hw": parts[5], "hw_thermal": parts[6], "sw_thermal": parts[7], "sw_power": parts[8]})
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hw_thermal", "hw_thermal_slowdown"),
                          ("sw_thermal", "sw_thermal_slowdown"), ("sw_power", "sw_power_cap")):
            if any(r[key].lower() == "active" for r in rows):
                reasons.append(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r["power"] for r in rows)}


def camera_setup():
    from paper_1803_08320_gb300 import malbec as mb
    from paper_1803_08320_gb300 import workloads as W

    cw = W.camera()
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    return cw, cam


def cpu_baseline(seconds: float = 12.0, max_seconds: float = 30.0) -> dict:
    """The oracle, untuned, on this host's cores: seeded random pixels of the
    same camera traced until about `seconds` of wall time have been spent."""
    import numpy as np

    import oracle

    cw, _ = camera_setup()
    rng = np.random.default_rng(20260)
    t_term = oracle.make_term(cw.term.eps_hor, cw.term.r_esc, cw.term.n_steps_cap, cw.term.dl, cw.term.dl_r_scale)
    steps = 0
    rays = 0
    threads = 0
    t0 = time.perf_counter()
    while True:
        pix = rng.choice(cw.n, 2048, replace=False)
        ics = oracle.camera_ics(cw.M, cw.a, cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny, pix)
        t1 = time.perf_counter()
        out = oracle.trace_many(cw.M, cw.a, ics, t_term, nthreads=0)
        steps += int(out["steps"].sum())
        rays += len(pix)
        threads = out["threads"]
        el = time.perf_counter() - t0
        if el >= seconds or el >= max_seconds:
            break
        del t1
    el = time.perf_counter() - t0
    return {"value": steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{rays} seeded random pixels of the {cw.nx}x{cw.ny} camera ({steps} RK4 steps, "
                      f"{el:.1f} s incl. initial-data construction), OpenMP over rays"}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cb = cpu_baseline(seconds=max(3.0, 10.0 * (args.steps / max(args.steps, 1))))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def load_traffic(kind: str):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except ValueError:
        return None
    ent = d.get(kind)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def run_profile_case(args) -> None:
    """The same camera at 512 x 512 (a quarter of the rays, same physics):
    small enough for a multi-pass ncu capture to end in seconds."""
    import torch

    from paper_1803_08320_gb300 import build as _b
    from paper_1803_08320_gb300 import malbec as mb
    from paper_1803_08320_gb300 import workloads as W

    _b.build()
    cw = W.camera(nx=512, ny=512)
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    prec = "fp64" if args.profile_case == "camera_fp64" else "fp32_mixed"
    for _ in range(max(1, args.steps)):
        res = mb.trace_camera(cw.M, cw.a, cam, cw.term, prec)
    torch.cuda.synchronize()
    steps = int(res["steps"].to(torch.int64).sum().item())
    print(json.dumps({"profile_case": args.profile_case, "rays": cw.n, "rk4_steps": steps}))


def timed_renders(mb, cw, cam, precision, K, stream, flush, out=None, host_out=None):
    """K renders, each bracketed by CUDA events on the launching stream; the L2
    is flushed (256 MB write) before each, outside the events."""
    import torch

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.zero_()
        evs[k][0].record(stream)
        res = mb.trace_camera(cw.M, cw.a, cam, cw.term, precision, stream=stream, out=out)
        if host_out is not None:
            host_out.copy_(res["buffer"], non_blocking=True)
        evs[k][1].record(stream)
    stream.synchronize()
    return [s.elapsed_time(e) for s, e in evs], res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="malbec", choices=["malbec", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", choices=["camera_fp64", "camera_mixed"], default=None,
                    help="small case for ncu: a 512x512 render of the same camera, --steps times")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1803_08320_gb300 import build as _b
    from paper_1803_08320_gb300 import malbec as mb

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    _b.build()
    stream = torch.cuda.Stream()
    cw, cam = camera_setup()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peak64 = mb.measure_fma_peak("fp64")
    peak32 = mb.measure_fma_peak("fp32_mixed")

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    with torch.cuda.stream(stream):
        L = mb.camera_layout(cam)
        out = torch.empty(L.total, dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            mb.trace_camera(cw.M, cw.a, cam, cw.term, "fp64", stream=stream, out=out)
        stream.synchronize()
        # ---------------- FP64 device-resident timing (the headline)
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clocks:
            times64, res = timed_renders(mb, cw, cam, "fp64", args.steps, stream, flush, out=out)
        torch.cuda.synchronize()
        barrier()
        steps_per_render = int(res["steps"].to(torch.int64).sum().item())
        st = res["steps"].to(torch.float64)
        step_dist = {"mean": float(st.mean().item()), "p99": float(torch.quantile(st[::16], 0.99).item()),
                     "max": int(res["steps"].max().item()),
                     "fates": {k: int((res["fate"] == v).sum().item()) for k, v in
                               (("captured", 1), ("escaped", 2), ("capped", 3), ("nonfinite", 4))}}
        fate64 = res["fate"].clone()
        theta64, phi64 = res["theta"].clone(), res["phi"].clone()
        t_total = max_over_ranks(sum(times64) / 1e3)
        value = world * steps_per_render * args.steps / t_total
        ms_per_step = 1e3 * t_total / args.steps

        # ---------------- FP32_MIXED, same protocol
        for _ in range(args.warmup):
            mb.trace_camera(cw.M, cw.a, cam, cw.term, "fp32_mixed", stream=stream, out=out)
        barrier()
        torch.cuda.synchronize()
        times32, res32 = timed_renders(mb, cw, cam, "fp32_mixed", args.steps, stream, flush, out=out)
        torch.cuda.synchronize()
        barrier()
        steps32 = int(res32["steps"].to(torch.int64).sum().item())
        t32 = max_over_ranks(sum(times32) / 1e3)
        value32 = world * steps32 * args.steps / t32
        f32 = res32["fate"]
        agree = float((f32 == fate64).float().mean().item())
        esc = (fate64 == mb.FATE_ESCAPED) & (f32 == mb.FATE_ESCAPED)
        dth = (res32["theta"][esc] - theta64[esc]).abs()
        dph = (res32["phi"][esc] - phi64[esc]).abs()
        dth, dph = dth[torch.isfinite(dth)], dph[torch.isfinite(dph)]

        # ---------------- end to end: the C-ABI render + device->host copy of the image
        host_out = torch.empty(L.total, dtype=torch.uint8, pin_memory=True)
        barrier()
        torch.cuda.synchronize()
        times_e2e, _ = timed_renders(mb, cw, cam, "fp64", args.steps, stream, flush, out=out, host_out=host_out)
        torch.cuda.synchronize()
        barrier()
        t_e2e = max_over_ranks(sum(times_e2e) / 1e3)
        value_e2e = world * steps_per_render * args.steps / t_e2e

    cl = clocks.summary()
    flops = FLOPS_PER_STEP["kerr"] * steps_per_render
    achieved = flops / (statistics.mean(times64) / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_step": cw.n, "rk4_steps_per_render": steps_per_render,
                   "steps_per_ray": step_dist,
                   "l2": "flushed by a 256 MB device write before every timed render (outside the events)",
                   "parallelism": f"replicas x{world} (one full render per GPU)"},
        "gpu_launches": args.steps,
        "clocks": {"sm_mhz": cl["sm_mhz"], "sm_max_mhz": cl["sm_max_mhz"], "reasons": cl["reasons"],
                   "samples": cl["samples"]},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak64, "unit": "GFLOP/s (FP64)",
                     "frac": achieved / peak64, "traffic": load_traffic("camera_fp64"),
                     "peak_note": "measured FP64 FMA loop on this GPU (malbec_measure_fma_peak), of measured",
                     "flops_per_rk4_step": FLOPS_PER_STEP["kerr"],
                     "plus_per_rk4_step": {"div": DIV_PER_STEP, "sincos": SINCOS_PER_STEP}},
        "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(L.total),
                "note": "malbec_trace_camera + copy of the image (fate, steps, theta, phi) to pinned host memory; "
                        "the rays are built on the device from the camera description passed by value"},
        "fp32_mixed": {"value": value32, "unit": UNIT, "ms_per_step": 1e3 * t32 / args.steps,
                       "speedup_vs_fp64": value32 / value, "fate_agreement_vs_fp64": agree,
                       "escaped_theta_max_abs_err": float(dth.max().item()) if dth.numel() else None,
                       "escaped_phi_max_abs_err": float(dph.max().item()) if dph.numel() else None,
                       "escaped_theta_median_abs_err": float(dth.median().item()) if dth.numel() else None,
                       "roofline": {"bound": "alu", "peak": peak32, "unit": "GFLOP/s (FP32)",
                                    "achieved_fp32_equiv": FLOPS_PER_STEP["kerr"] * steps32 /
                                    (statistics.mean(times32) / 1e3) / 1e9,
                                    "frac": FLOPS_PER_STEP["kerr"] * steps32 / (statistics.mean(times32) / 1e3)
                                    / 1e9 / peak32}},
    }
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

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
import dataclasses
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
KERNEL_SOURCES = ["geodesic.cuh", "camera.cuh", "fp32pair.cuh", "trace_kernel.cuh", "trace.cu", "trace_dopri.cu"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1803_08320_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# algorithmic flops per RK4 step, counted from the kernel source expressions
# (FMA = 2, add/mul = 1, a product or sum written once and reused counted
# once): 89 per Kerr right-hand side of the geodesic form (42 products, 20
# FMA, 7 sums: the contraction written through q = 2Mr/rho^2 and
# v = u^t - a sin^2 u^phi), 42 per Schwarzschild one, 102 for the RK4 stage
# points and weighted sums; the
# canonical form (eq. Ham): 72 per Kerr right-hand side, 74 for its RK4
# (p_t, p_ph fixed); the 3+1 form: 65 for Kerr's lapse, shift, 3-metric and
# their logarithmic derivatives plus 34 for the 3+1 right-hand side, the same
# 74 for its RK4.  Listed separately per step: 4 reciprocals (a hardware
# estimate and 3 FMA each), 1 sincos and 3 stage-angle rotations (angle
# addition with short Taylor series, 17 FP64 operations each: 3 products, 14 FMA).
FLOPS_PER_STEP = {"kerr": 4 * 89 + 102, "schw": 4 * 42 + 102, "kerr_canonical": 4 * 72 + 74,
                  "kerr_adm": 4 * (65 + 34) + 74,
                  # Dormand-Prince 5(4) attempt: 6 Kerr right-hand sides, 272 for
                  # the six stage combinations, 72 + 16 for the stage points and
                  # the fifth-order result, 6 for the stage-angle offsets, 96 for
                  # the error estimate, 33 for the error norm (its 8 divisions,
                  # sqrt and log2 listed apart, like the 6 reciprocals, 1 sincos
                  # and 6 stage-angle rotations)
                  "kerr_dopri5": 6 * 89 + 272 + 72 + 16 + 6 + 96 + 33}
PLUS_PER_STEP = {"reciprocal": 4, "sincos": 1, "stage_angle_rotation": 3}


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


def cpu_model() -> str:
    """The host CPU's model name (Linux /proc/cpuinfo; 'unknown' elsewhere)."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


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
    # one host core, for comparison with the paper's sequential C (Sec. 6.4)
    pix = rng.choice(cw.n, 256, replace=False)
    ics = oracle.camera_ics(cw.M, cw.a, cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny, pix)
    t1 = time.perf_counter()
    out1 = oracle.trace_many(cw.M, cw.a, ics, t_term, nthreads=1)
    single = int(out1["steps"].sum()) / (time.perf_counter() - t1)
    return {"value": steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{rays} seeded random pixels of the {cw.nx}x{cw.ny} camera ({steps} RK4 steps, "
                      f"{el:.1f} s incl. initial-data construction), OpenMP over rays",
            "single_thread_value": single, "cpu_model": cpu_model()}


REFERENCE_PIXELS_PER_STEP = 16384


def run_reference(args) -> None:
    """The oracle as it stands, on this host's cores: every step traces a
    fresh seeded sample of REFERENCE_PIXELS_PER_STEP pixels of the same camera
    (W warm-up samples, then K timed ones)."""
    import numpy as np

    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cw, _ = camera_setup()
    t_term = oracle.make_term(cw.term.eps_hor, cw.term.r_esc, cw.term.n_steps_cap, cw.term.dl, cw.term.dl_r_scale)
    rng = np.random.default_rng(20261)

    def sample():
        pix = rng.choice(cw.n, REFERENCE_PIXELS_PER_STEP, replace=False)
        t0 = time.perf_counter()
        ics = oracle.camera_ics(cw.M, cw.a, cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny, pix)
        out = oracle.trace_many(cw.M, cw.a, ics, t_term, nthreads=0)
        return int(out["steps"].sum()), time.perf_counter() - t0, out["threads"]

    for _ in range(args.warmup):
        sample()
    steps = secs = 0
    threads = 0
    for _ in range(args.steps):
        s, t, threads = sample()
        steps += s
        secs += t
    value = steps / secs
    cb = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
          "sample": f"{args.steps} x {REFERENCE_PIXELS_PER_STEP} seeded random pixels of the {cw.nx}x{cw.ny} camera "
                    f"({steps} RK4 steps in {secs:.1f} s incl. initial data), OpenMP over rays"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"]}, "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def load_traffic(kind: str, field: str = "dram_bytes_per_launch"):
    """A figure of the committed ncu summary (dram bytes per launch, FP64 pipe
    utilisation), if it was taken on the current kernel source (else None)."""
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
    return ent.get(field)


def run_profile_case(args) -> None:
    """The same camera at 512 x 512 (a quarter of the rays, same physics):
    small enough for a multi-pass ncu capture to end in seconds; the
    *_1024 cases are the benchmark's own 1024 x 1024 image (for captures of
    a few metrics)."""
    import torch

    from paper_1803_08320_gb300 import build as _b
    from paper_1803_08320_gb300 import malbec as mb
    from paper_1803_08320_gb300 import workloads as W

    _b.build()
    if args.profile_case == "traj_mixed":
        # 65536 bound orbits x 1000 steps, a sample every step, FP32_MIXED:
        # 2.1 GB of trajectory on the device
        wl = W.bound(n=1 << 16, n_steps=1000)
        ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, wl.n)
        t = W.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=1000, dl=0.02)
        for _ in range(max(1, args.steps)):
            res = mb.trace(wl.M, 0.0, ics, t, mode=mb.OUT_STRIDED, stride=1, precision="fp32_mixed",
                           a_per_ray=spins)
        torch.cuda.synchronize()
        steps = int(res["steps"].to(torch.int64).sum().item())
        print(json.dumps({"profile_case": args.profile_case, "rays": wl.n, "rk4_steps": steps}))
        return
    side = 1024 if args.profile_case.endswith("1024") else 512
    cw = W.camera(nx=side, ny=side)
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    prec = "fp32_mixed" if "mixed" in args.profile_case else "fp64"
    form = {"camera_canonical": mb.FORM_HAMILTONIAN, "camera_adm": mb.FORM_ADM}.get(args.profile_case,
                                                                                   mb.FORM_GEODESIC)
    term = mb.term_from(cw.term, form=form)
    if args.profile_case == "camera_dopri5":
        term = dataclasses.replace(mb.term_from(cw.term, method=mb.METHOD_DOPRI5, rtol=1e-9, atol=1e-9),
                                   dl=0.0, dl_r_scale=0.5)
    if args.profile_case == "camera_mixed_dopri5_1024":
        term = dataclasses.replace(mb.term_from(cw.term, method=mb.METHOD_DOPRI5, rtol=1e-6, atol=1e-6),
                                   dl=0.0, dl_r_scale=0.5)
    for _ in range(max(1, args.steps)):
        res = mb.trace_camera(cw.M, cw.a, cam, term, prec)
    torch.cuda.synchronize()
    steps = int(res["steps"].to(torch.int64).sum().item())
    print(json.dumps({"profile_case": args.profile_case, "rays": cw.n, "rk4_steps": steps}))


BUNDLE_FOV_HALF, BUNDLE_R_OBS = 25.0, 1000.0


def bundle_of(mb, kind: str, n: int, a: float, cap: int, incl: float, seed: int, side: int = 0):
    """One malbec_bundle from a workload item: a camera patch (the first n
    pixels of a side x side camera over +-25M, step 0.05 r) or a generic
    bound-orbit ensemble sampled in the kernel (dtau = 0.02)."""
    if kind == "camera":
        side = side or (math.isqrt(n - 1) + 1)
        t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=cap, dl=0.0, dl_r_scale=0.05)
        cam = mb.make_camera(BUNDLE_R_OBS, incl, BUNDLE_FOV_HALF, side, side)
        return mb.make_bundle(mb.BUNDLE_CAMERA, n, 1.0, a, t, camera=cam)
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=cap, dl=0.02)
    return mb.make_bundle(mb.BUNDLE_BOUND, n, 1.0, a, t, seed=seed)


def steps_of(views) -> int:
    return int(sum(int(v["steps"].to(__import__("torch").int64).sum().item()) for v in views))


def run_bundles_case(mb, torch, stream, flush, count: int, precision: str, K: int, warmup: int,
                     autotune_every: int = 8, per_bundle_arm: bool = True, refine_full_list: bool = True) -> dict:
    """Uneven bundles (the first `count` of the 4096-bundle list): one
    persistent launch replayed from a CUDA graph after autotuning, against
    one launch per bundle on the same stream.  Each timed pass is bracketed
    by CUDA events on the launching stream, with the L2 flushed before it."""
    from paper_1803_08320_gb300 import workloads as W

    specs = W.bundles()[:count]
    bundles = [bundle_of(mb, s.kind, s.n, s.a, s.cap, s.incl, s.seed) for s in specs]
    views = mb.attach_outputs(bundles, precision)
    rays = sum(s.n for s in specs)

    # autotune on every `autotune_every`-th bundle (same size and cap mix),
    # then record the full plan with the winning launch configuration
    saved = mb.get_launch_config().as_dict()
    sub = bundles[::autotune_every]
    t_at = time.perf_counter()
    sub_plan = mb.Plan(sub, precision)
    best = sub_plan.autotune(stream=stream)
    torch.cuda.synchronize()
    sub_plan.close()
    t_at = time.perf_counter() - t_at
    # second stage on the full list: the subset's choice against the same
    # configuration with one more block per SM (the subset has fewer rays in
    # flight, so it can prefer fewer resident warps than the full list), one
    # replay each after a warm-up replay; the faster one is timed below
    refine = {}
    if refine_full_list and count > len(sub):
        alt = dict(best, blocks_per_sm=best["blocks_per_sm"] + 1)
        for name, cfg in (("subset_choice", best), ("one_more_block_per_sm", alt)):
            mb.set_launch_config(**cfg)
            p2 = mb.Plan(bundles, precision)
            mb.set_launch_config(**saved)
            with torch.cuda.stream(stream):
                p2.launch(stream=stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                e0.record(stream)
                p2.launch(stream=stream)
                e1.record(stream)
                stream.synchronize()
            p2.close()
            refine[name] = {"config": cfg, "seconds": e0.elapsed_time(e1) / 1e3}
        if refine["one_more_block_per_sm"]["seconds"] < refine["subset_choice"]["seconds"]:
            best = refine["one_more_block_per_sm"]["config"]
    mb.set_launch_config(**best)
    plan = mb.Plan(bundles, precision)
    mb.set_launch_config(**saved)

    def timed(fn, k):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            flush.zero_()
            evs[i][0].record(stream)
            fn()
            evs[i][1].record(stream)
        stream.synchronize()
        return [s.elapsed_time(e) / 1e3 for s, e in evs]

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            plan.launch(stream=stream)
        stream.synchronize()
        t_plan = timed(lambda: plan.launch(stream=stream), K)
        steps_plan = steps_of(views)
        fates_plan = [v["fate"].clone() for v in views]

        def per_bundle():
            for b in bundles:
                mb.trace_bundles([b], precision, stream=stream)

        if per_bundle_arm:
            # the kernel is already warm: one small launch before the timed passes
            mb.trace_bundles([min(bundles, key=lambda b: b.n)], precision, stream=stream)
            stream.synchronize()
            t_each = timed(per_bundle, K)
            steps_each = steps_of(views)
            agree = sum(int((v["fate"] == f).sum().item()) for v, f in zip(views, fates_plan)) / rays
    plan.close()
    v_plan = steps_plan / statistics.mean(t_plan)
    each = None
    if per_bundle_arm:
        v_each = steps_each / statistics.mean(t_each)
        each = {"value": v_each, "unit": UNIT, "ms_per_pass": 1e3 * statistics.mean(t_each),
                "gpu_launches_per_pass": count, "rk4_steps_per_pass": steps_each, "fate_agreement_with_graph": agree}
    return {"bundles": count, "rays": rays, "precision": precision, "rk4_steps_per_pass": steps_plan,
            "persistent_graph": {"value": v_plan, "unit": UNIT, "ms_per_pass": 1e3 * statistics.mean(t_plan),
                                 "gpu_launches_per_pass": 1},
            "one_launch_per_bundle": each,
            "speedup": v_plan / each["value"] if each else None,
            "autotune": {"best": best, "on_bundles": len(sub), "seconds": t_at, "full_list_refinement": refine},
            "l2": "flushed before every timed pass (outside the events)"}


def drift_stats(inv0, inv1) -> dict:
    """Per-particle |inv1 - inv0| / max(|inv0|, 1) of E, L_z, Q and the norm."""
    import numpy as np

    d = np.abs(inv1 - inv0) / np.maximum(np.abs(inv0), 1.0)
    out = {}
    for i, name in enumerate(("E", "Lz", "Q", "norm")):
        x = d[i][np.isfinite(d[i])]
        out[name] = {"median": float(np.median(x)), "p99": float(np.quantile(x, 0.99)), "max": float(x.max()),
                     "frac_le_1e-6": float((x <= 1e-6).mean()), "nonfinite": int((~np.isfinite(d[i])).sum())}
    return out


def cpu_baseline_bound(wl, idx):
    """The oracle on the 1024-particle subsample of the generic bound-orbit
    workload (indices k * 1024), on this host's cores: its timing, and its
    final states for the error statement of the GPU results."""
    import numpy as np

    import oracle

    t = oracle.make_term(wl.term.eps_hor, wl.term.r_esc, wl.term.n_steps_cap, wl.term.dl, wl.term.dl_r_scale)
    ys, spins, _ = oracle.bound_samples(wl.M, wl.a_max, wl.seed, idx)
    t0 = time.perf_counter()
    ref = oracle.trace_many(wl.M, 0.0, ys, t, a_per_ray=spins, nthreads=0)
    el = time.perf_counter() - t0
    steps = int(ref["steps"].sum())
    return ref, {"value": steps / el, "unit": UNIT, "cores": ref["threads"], "kind": "oracle",
                 "sample": f"{len(idx)} particles (indices k*1024), {steps} RK4 steps in {el:.1f} s, OpenMP over "
                           f"particles"}


def run_bound_case(mb, torch, stream, flush, n: int, n_steps: int, precisions, with_oracle: bool = True) -> dict:
    """Generic bound Kerr orbits (spin U[0, 0.998], r_p in [ISCO + 0.5M, 10M],
    e U[0, 0.7], inclination U[0, pi]; dtau = 0.02): one timed pass per
    precision (CUDA events on the launching stream, L2 flushed before it;
    warm-up: the same launch with a 1000-step cap), conserved-quantity drift
    per particle, and on the subsample k * 1024 the final state against the
    oracle."""
    import numpy as np

    from paper_1803_08320_gb300 import workloads as W

    wl = W.bound(n=n, n_steps=n_steps)
    warm = W.Termination(eps_hor=wl.term.eps_hor, r_esc=wl.term.r_esc, n_steps_cap=1000, dl=wl.term.dl)
    with torch.cuda.stream(stream):
        ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, n, stream=stream)
    stream.synchronize()
    idx = np.arange(0, n, 1024)[:1024]
    ref = cb = None
    if with_oracle:
        ref, cb = cpu_baseline_bound(wl, idx)
    res = {"particles": n, "rk4_steps_cap": n_steps, "dtau": wl.term.dl}
    for prec in precisions:
        L = mb.out_layout(mb.OUT_FINAL, prec, n, n_steps, 0)
        out = torch.empty(L.total, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(3):
                mb.trace(wl.M, 0.0, ics, warm, precision=prec, a_per_ray=spins, stream=stream, out=out)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = mb.trace(wl.M, 0.0, ics, wl.term, precision=prec, a_per_ray=spins, stream=stream, out=out)
            e1.record(stream)
        stream.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        steps = int(r["steps"].to(torch.int64).sum().item())
        ent = {"value": steps / sec, "unit": UNIT, "seconds": sec, "rk4_steps": steps,
               "fates": fate_counts(mb, r["fate"]),
               "drift_all_particles": drift_stats(r["inv0"].cpu().numpy(), r["inv1"].cpu().numpy())}
        capped = ((r["fate"] & mb.FATE_MASK) == mb.FATE_CAPPED).cpu().numpy()
        ent["drift_capped_particles"] = drift_stats(r["inv0"].cpu().numpy()[:, capped],
                                                    r["inv1"].cpu().numpy()[:, capped])
        ent["drift_note"] = ("particles that end before the cap are orbits that pass next to the polar axis, where "
                             "fixed-step RK4 in Boyer-Lindquist coordinates is ill-conditioned in any precision")
        if ref is not None:
            y = r["y"].cpu().numpy()[:, idx]
            with np.errstate(invalid="ignore"):
                rel = np.abs(y - ref["y"]) / np.maximum(np.abs(ref["y"]), 1.0)
            worst = np.where(np.isfinite(rel), rel, np.inf).max(axis=0)
            ent["subsample_vs_oracle"] = {
                "particles": len(idx), "median_max_rel": float(np.median(worst)),
                "frac_within_1e-9": float((worst <= 1e-9).mean()), "frac_within_1e-6": float((worst <= 1e-6).mean()),
                "fate_agreement": float((r["fate"].cpu().numpy()[idx] == ref["fate"]).mean()),
                "oracle_drift": drift_stats(ref["inv0"], ref["inv1"])}
        res[prec] = ent
        del out, r
    if "fp64" in res and "fp32_mixed" in res:
        res["mixed_speedup_vs_fp64"] = res["fp32_mixed"]["value"] / res["fp64"]["value"]
    if cb is not None:
        res["cpu_baseline"] = cb
    return res


# The paper's timing experiment (Sec. 6.4, its two tables of GPU and CPU
# run times): Kerr a = 0.5M, RK4 with h = 0.1, t_f = 1000 (10^4 steps, t_f
# read as proper time), N random timelike geodesics; its GPU run times in
# seconds, without and with per-step output to disk.
PAPER_N = (10, 100, 500, 1000, 5000, 10000, 50000)
PAPER_GPU_S_NO_OUTPUT = {10: 2.16987, 100: 2.301033, 500: 4.628749, 1000: 4.63499, 5000: 13.598218,
                         10000: 27.066675}
PAPER_GPU_S_WITH_OUTPUT = {10: 60 * 0.0545956, 100: 60 * 0.11868735, 500: 60 * 0.3829293, 1000: 60 * 0.66657395,
                           5000: 60 * 3.543259, 10000: 60 * 7.14927418, 50000: 60 * 35.6253648}


def run_paper_case(mb, torch, stream, stride: int = 10) -> dict:
    """The paper's timing experiment on this GPU, FP64: for each N, the
    generic bound-orbit sampler with the spin fixed at 0.5 gives the N
    initial states (the paper's are unspecified random timelike geodesics),
    traced 10^4 steps of h = 0.1 (a) with the final state only and (b) with
    the trajectory every `stride` steps copied to pinned host memory (the
    paper writes ASCII at every step).  CUDA events on the launching stream;
    (b) includes the device-to-host copy."""
    from paper_1803_08320_gb300 import workloads as W

    term = W.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=10_000, dl=0.1)
    n_max = max(PAPER_N)
    ics_all, _, _ = mb.ic_bound(1.0, 0.5, W.SEED_BASE + 6, n_max, spin_fixed=True)
    Lmax = mb.out_layout(mb.OUT_STRIDED, "fp64", n_max, term.n_steps_cap, stride)
    out = torch.empty(Lmax.total, dtype=torch.uint8, device="cuda")
    host = torch.empty(Lmax.total, dtype=torch.uint8, pin_memory=True)
    rows = []
    with torch.cuda.stream(stream):
        mb.trace(1.0, 0.5, ics_all[:, :10].contiguous(), term, precision="fp64", stream=stream, out=out)
        for n in PAPER_N:
            ics = ics_all[:, :n].contiguous()
            row = {"n": n}
            for mode in ("final", "strided"):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                stream.synchronize()
                e0.record(stream)
                if mode == "final":
                    r = mb.trace(1.0, 0.5, ics, term, precision="fp64", stream=stream, out=out)
                    nbytes = 0
                else:
                    L = mb.out_layout(mb.OUT_STRIDED, "fp64", n, term.n_steps_cap, stride)
                    r = mb.trace(1.0, 0.5, ics, term, mode=mb.OUT_STRIDED, stride=stride, precision="fp64",
                                 stream=stream, out=out)
                    host[:L.total].copy_(out[:L.total], non_blocking=True)
                    nbytes = int(L.total)
                e1.record(stream)
                stream.synchronize()
                sec = e0.elapsed_time(e1) / 1e3
                steps = int(r["steps"].to(torch.int64).sum().item())
                row[mode] = {"seconds": sec, "steps_per_s": steps / sec, "d2h_bytes": nbytes}
            # the same rays in FP32_MIXED, final state only: the latency of a
            # small batch is that of one lane's sequence of steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            e0.record(stream)
            r = mb.trace(1.0, 0.5, ics, term, precision="fp32_mixed", stream=stream, out=out)
            e1.record(stream)
            stream.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            steps = int(r["steps"].to(torch.int64).sum().item())
            row["final_fp32_mixed"] = {"seconds": sec, "steps_per_s": steps / sec,
                                       "us_per_step_of_one_ray": 1e6 * sec / term.n_steps_cap}
            row["final"]["us_per_step_of_one_ray"] = 1e6 * row["final"]["seconds"] / term.n_steps_cap
            p0, p1 = PAPER_GPU_S_NO_OUTPUT.get(n), PAPER_GPU_S_WITH_OUTPUT.get(n)
            row["paper_gpu_seconds"] = {"no_output": p0, "with_ascii_output": p1}
            row["speedup_vs_paper_gpu"] = {"no_output": p0 / row["final"]["seconds"] if p0 else None,
                                           "with_output": p1 / row["strided"]["seconds"] if p1 else None}
            rows.append(row)
    return {"a": 0.5, "h": 0.1, "rk4_steps_per_ray": 10_000, "trajectory_stride": stride,
            "precision": "fp64 (and fp32_mixed, final state only)",
            "rows": rows,
            "paper_hardware": "GTX 960M (Maxwell), CUDA 7.5; the paper's numbers are context, not a target"}


def run_trajectory_case(mb, torch, stream, flush, n: int = 1 << 17, n_steps: int = 2000) -> dict:
    """Trajectory-write mode (OUT_STRIDED) against the final-state mode on
    generic bound orbits (the config-3 sampler, dtau = 0.02), FP64 and
    FP32_MIXED, strides 10 and 1: steps/s and the bytes of trajectory samples
    written per second (64 B per FP64 sample, 32 B per FP32 one) against the
    measured HBM copy bandwidth.  One timed launch per row after an identical
    warm-up launch, L2 flushed before it, CUDA events on the stream."""
    from paper_1803_08320_gb300 import workloads as W

    wl = W.bound(n=n, n_steps=n_steps)
    ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, n, stream=stream)
    t = W.Termination(eps_hor=wl.term.eps_hor, r_esc=wl.term.r_esc, n_steps_cap=n_steps, dl=wl.term.dl)
    hbm = None
    peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks):
        hbm = json.load(open(peaks)).get("hbm_gbs")
    rows = []
    for prec in ("fp64", "fp32_mixed"):
        elem = 8 if prec == "fp64" else 4
        for mode, stride in ((mb.OUT_FINAL, 0), (mb.OUT_STRIDED, 10), (mb.OUT_STRIDED, 1)):
            L = mb.out_layout(mode, prec, n, n_steps, stride)
            out = torch.empty(L.total, dtype=torch.uint8, device="cuda")
            with torch.cuda.stream(stream):
                mb.trace(wl.M, 0.0, ics, t, mode=mode, stride=stride, precision=prec, a_per_ray=spins,
                         stream=stream, out=out)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                e0.record(stream)
                r = mb.trace(wl.M, 0.0, ics, t, mode=mode, stride=stride, precision=prec, a_per_ray=spins,
                             stream=stream, out=out)
                e1.record(stream)
                stream.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            steps = int(r["steps"].to(torch.int64).sum().item())
            nbytes = n * int(L.n_samples) * 8 * elem if mode == mb.OUT_STRIDED else 0
            row = {"precision": prec, "mode": "strided" if mode == mb.OUT_STRIDED else "final", "stride": stride,
                   "seconds": sec, "steps_per_s": steps / sec, "trajectory_bytes": nbytes,
                   "write_gb_per_s": nbytes / sec / 1e9}
            if hbm:
                row["frac_of_hbm_copy"] = nbytes / sec / 1e9 / hbm
            rows.append(row)
            del out, r
            torch.cuda.empty_cache()
    return {"particles": n, "rk4_steps_cap": n_steps, "dtau": wl.term.dl, "hbm_gbs_measured": hbm, "rows": rows}


def drift_summary(mb, torch, r) -> dict:
    """Median and p99 of |inv1 - inv0| (E, L_z, Q, g(u,u)) over the rays that
    did not end non-finite."""
    ok = (r["fate"] & mb.FATE_MASK) != mb.FATE_NONFINITE
    out = {}
    for c, nm in enumerate(("E", "Lz", "Q", "norm")):
        d = (r["inv1"][c] - r["inv0"][c]).abs()[ok]
        d = d[torch.isfinite(d)]
        out[nm] = {"median": float(d.median().item()), "p99": float(torch.quantile(d, 0.99).item())}
    out["nonfinite"] = int((~ok).sum().item())
    return out


def run_integrators_case(mb, torch, stream, flush, K: int, warmup: int) -> dict:
    """Work against accuracy on the camera workload (Kerr a = 0.9, 1024^2):
    RK4 with the camera's step rule against Dormand-Prince 5(4) at several
    tolerances (steps at most 0.5 r).  Per configuration: ms per render (CUDA
    events, L2 flushed, K renders after `warmup`), RK4 steps or attempts per
    ray, right-hand sides per ray, and the drift of the flow's invariants on
    every 16th pixel traced as a state array."""
    import numpy as np

    from paper_1803_08320_gb300 import workloads as W

    cw = W.camera()
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    L = mb.camera_layout(cam)
    out = torch.empty(L.total, dtype=torch.uint8, device="cuda")
    ics_s = mb.ic_camera(cw.M, cw.a, cam, np.arange(0, cw.n, 16), stream=stream)
    configs = [("rk4_h0.05r", mb.term_from(cw.term))]
    for tol in (1e-6, 1e-7, 1e-8, 1e-9, 1e-10):
        t = mb.term_from(cw.term, method=mb.METHOD_DOPRI5, rtol=tol, atol=tol)
        configs.append((f"dopri5_tol{tol:g}", dataclasses.replace(t, dl=0.0, dl_r_scale=0.5)))
    rows = {}
    for name, t in configs:
        run = CameraRun(cw.M, cw.a, t)
        for _ in range(warmup):
            mb.trace_camera(cw.M, cw.a, cam, t, "fp64", stream=stream, out=out)
        torch.cuda.synchronize()
        times, res = timed_renders(mb, run, cam, "fp64", K, stream, flush, out=out)
        steps = int(res["steps"].to(torch.int64).sum().item())
        rhs = (4.0 * steps if t.method == mb.METHOD_RK4 else 6.0 * steps + cw.n) / cw.n
        rr = mb.trace(cw.M, cw.a, ics_s, t, precision="fp64", stream=stream)
        torch.cuda.synchronize()
        rows[name] = {"ms_per_render": statistics.mean(times), "steps_or_attempts_per_ray": steps / cw.n,
                      "rhs_per_ray": rhs, "rays_per_s": cw.n / (statistics.mean(times) / 1e3),
                      "invariant_drift_65536_pixels": drift_summary(mb, torch, rr)}
    return {"workload": "kerr_camera_a0.9_1024x1024", "renders": K, "rows": rows}


def cw_steps_per_s(row) -> float:
    return row["steps_or_attempts_per_ray"] * row["rays_per_s"]


def q_ratio(finals):
    """The paper's self-convergence ratio Q = |y_h - y_h/2| / |y_h/2 - y_h/4|
    (Sec. 6.3, eq. Qt; 2^4 for a fourth-order method), per ray from the max
    over state components; rays with a non-finite or vanishing difference
    are left out."""
    import numpy as np

    d1 = np.abs(finals[0] - finals[1]).max(axis=0)
    d2 = np.abs(finals[1] - finals[2]).max(axis=0)
    ok = np.isfinite(d1) & np.isfinite(d2) & (d2 > 1e-12)
    q = d1[ok] / d2[ok]
    return {"rays": int(ok.sum()), "of": int(d1.size), "median": float(np.median(q)) if q.size else None,
            "frac_13_19": float(np.mean((q > 13.0) & (q < 19.0))) if q.size else None}


def run_convergence_case(mb, torch, stream) -> dict:
    """The paper's self-convergence test (Sec. 6.3) on the GPU, FP64, for the
    three physics configurations: each traced with fixed steps h, h/2, h/4 to
    the same affine parameter (camera rays with a fixed step, which is what
    the test is defined for, from their camera initial states)."""
    import numpy as np

    from paper_1803_08320_gb300 import workloads as W

    out = {}
    cases = []
    # config 1's circular orbits with a radial kick u^r = 0.01: an exact
    # circular orbit is a fixed point of the right-hand side in (r, theta, u),
    # which RK4 follows exactly up to rounding, so Q needs some dynamics
    wl = W.circular()
    ic1 = mb.ic_circular(1.0, 0.0, wl.radii)
    ic1[5] = 0.01
    cases.append(("1_schwarzschild_circular_1024_kicked", 0.0, ic1, None, (1.6, 0.8, 0.4), 800.0))
    cw = W.camera(nx=128, ny=128)
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    cases.append(("2_kerr_a0.9_camera_128x128", cw.a, mb.ic_camera(cw.M, cw.a, cam, np.arange(cw.n)), None,
                  (0.2, 0.1, 0.05), 1040.0))
    bw = W.bound()
    ics, spins, _ = mb.ic_bound(bw.M, bw.a_max, bw.seed, 1024)
    cases.append(("3_kerr_generic_bound_1024", 0.0, ics, spins, (0.1, 0.05, 0.025), 100.0))
    with torch.cuda.stream(stream):
        for name, a, y0, spins, hs, lam_end in cases:
            finals = []
            for h in hs:
                t = W.Termination(eps_hor=0.01, r_esc=1e9, n_steps_cap=int(round(lam_end / h)), dl=h)
                r = mb.trace(1.0, a, y0, t, precision="fp64", stream=stream, a_per_ray=spins)
                stream.synchronize()
                keep = (r["fate"] & mb.FATE_MASK) == mb.FATE_CAPPED
                y = r["y"].clone()
                y[:, ~keep] = float("nan")
                finals.append(y.cpu().numpy())
            out[name] = dict(q_ratio(finals), h=list(hs), affine_end=lam_end)
    return out


def serving_bundle(mb, r):
    return bundle_of(mb, r.kind, r.n, r.a, r.cap, r.incl, r.seed, side=r.side)


def run_serving_case(mb, torch, rate: float, n_req: int, precision: str, budget: int = 150 * 10**9,
                     timeout_s: float = 300.0, stretch: float = 1.0, baseline_streams=(1,)) -> dict:
    """Poisson arrivals at `rate` req/s (the first n_req of the seeded stream;
    with `stretch` > 1 the same requests arrive that many times further
    apart), replayed in wall-clock time against (a) the continuous-batching
    server and (b) one launch per request, in arrival order, round-robin on
    k streams for each k in `baseline_streams`.  Latency = scheduled arrival
    -> the host sees the job's results complete in HBM.  Throughput = all RK4
    steps / (first arrival -> last completion)."""
    from paper_1803_08320_gb300 import workloads as W

    reqs = W.serving(rate, duration=50.0 * n_req / rate)[:n_req]
    n_req = len(reqs)
    t_arr = [stretch * (r.t_arrival - reqs[0].t_arrival) for r in reqs]
    cams = sum(1 for r in reqs if r.kind == "camera")

    def summarise(lat, steps, span):
        lat = sorted(lat)
        q = lambda p: lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)]
        return {"p50_ms": 1e3 * q(0.50), "p99_ms": 1e3 * q(0.99), "mean_ms": 1e3 * statistics.mean(lat),
                "max_ms": 1e3 * lat[-1], "steps_per_s": steps / span, "makespan_s": span, "rk4_steps": steps}

    # (a) the server
    bundles = [serving_bundle(mb, r) for r in reqs]
    srv = mb.Server(hbm_budget=budget, max_active=1024, precision=precision, idle_timeout_s=0.002)
    done_at, ids = {}, {}
    i = 0
    t0 = time.perf_counter()
    while len(done_at) < n_req:
        now = time.perf_counter() - t0
        assert now < timeout_s, "serving run exceeded its time limit"
        while i < n_req and t_arr[i] <= now:
            ids[srv.submit(bundles[i])] = i
            i += 1
        for jid, k in list(ids.items()):
            if k not in done_at and srv.poll(jid):
                done_at[k] = time.perf_counter() - t0
    stats = srv.stats()
    steps = 0
    for jid in ids:
        v = srv.output(jid)
        steps += int(v["steps"].to(torch.int64).sum().item())
        srv.release(jid)
    srv.close()
    lat = [done_at[k] - t_arr[k] for k in range(n_req)]
    served = summarise(lat, steps, max(done_at.values()))
    served["gpu_launches"] = int(stats["kernel_launches"])

    # (b) one launch per request, round-robin on k streams
    singles = {}
    for k_streams in baseline_streams:
        streams = [torch.cuda.Stream() for _ in range(k_streams)]
        bundles = [serving_bundle(mb, r) for r in reqs]
        inflight, bufs, done_at = {}, [], {}
        i = 0
        t0 = time.perf_counter()
        while len(done_at) < n_req:
            now = time.perf_counter() - t0
            assert now < timeout_s, "one-launch-per-request run exceeded its time limit"
            while i < n_req and t_arr[i] <= now:
                st = streams[i % k_streams]
                with torch.cuda.stream(st):
                    (v,) = mb.attach_outputs([bundles[i]], precision)
                mb.trace_bundles([bundles[i]], precision, stream=st)
                ev = torch.cuda.Event()
                ev.record(st)
                inflight[i] = ev
                bufs.append(v)
                i += 1
            for k, ev in list(inflight.items()):
                if ev.query():
                    done_at[k] = time.perf_counter() - t0
                    del inflight[k]
        torch.cuda.synchronize()
        steps_b = steps_of(bufs)
        lat = [done_at[k] - t_arr[k] for k in range(n_req)]
        single = summarise(lat, steps_b, max(done_at.values()))
        single["gpu_launches"] = n_req
        single["streams"] = k_streams
        singles[k_streams] = single
    single = singles[baseline_streams[0]]
    span = max(t_arr[-1], 1e-9)
    out = {"rate_req_s": rate / stretch, "requests": n_req, "camera_requests": cams, "precision": precision,
           "arrival_span_s": span, "offered_req_s": n_req / span, "offered_steps_per_s": steps / span,
           "hbm_budget_bytes": budget, "continuous_batching": served, "one_launch_per_request": single,
           "p50_speedup": single["p50_ms"] / served["p50_ms"], "p99_speedup": single["p99_ms"] / served["p99_ms"],
           "throughput_ratio": served["steps_per_s"] / single["steps_per_s"]}
    if len(singles) > 1:
        out["one_launch_per_request_streams"] = {str(k): v for k, v in singles.items()}
    return out


def run_serving_low_load(mb, torch, saturated: dict, n_req: int, precision: str, utilization: float = 0.7) -> dict:
    """The same requests as a saturated run, arriving further apart so that
    the offered work (their RK4 steps per second of arrivals) is `utilization`
    of the continuous-batching throughput measured under saturation: latency
    below capacity, against one launch per request on 1 and 4 streams."""
    capacity = saturated["continuous_batching"]["steps_per_s"]
    stretch = max(1.0, saturated["offered_steps_per_s"] / (utilization * capacity))
    res = run_serving_case(mb, torch, rate=saturated["rate_req_s"], n_req=n_req, precision=precision,
                           stretch=stretch, baseline_streams=(1, 4))
    res["offered_utilization"] = res["offered_steps_per_s"] / capacity
    res["capacity_steps_per_s"] = capacity
    res["note"] = ("the requests of the saturated sample, arrival times stretched x%.2f so that the offered "
                   "work is %.0f%% of the saturated continuous-batching throughput" % (stretch, 100 * utilization))
    return res


def fate_counts(mb, fate) -> dict:
    """Rays per termination (fate & FATE_MASK) and how many of them carry the
    validity flag (FATE_DRIFTED: the norm g(u,u) drifted by more than
    NORM_DRIFT_TOL max(E^2, |g|); set on ESCAPED and CAPPED rays only)."""
    base = fate & mb.FATE_MASK
    flag = (fate & mb.FATE_DRIFTED) != 0
    out = {}
    for k, v in (("captured", 1), ("escaped", 2), ("capped", 3), ("nonfinite", 4)):
        sel = base == v
        out[k] = int(sel.sum().item())
        if v in (2, 3):
            out[k + "_drifted"] = int((sel & flag).sum().item())
    out["drifted_fraction"] = float(flag.float().mean().item())
    return out


def err_stats(torch, dth, dph) -> dict:
    """|FP32_MIXED - FP64| of the final (theta, phi) of rays both runs call
    ESCAPED without the validity flag: quantiles, maximum and the count above
    1e-6 rad.  The flag removes the rays whose norm a fixed step broke (passages
    next to the polar axis, ill-conditioned in both precisions), so the
    maximum is finite and describes rays with a trustworthy result."""
    out = {"rays": int(dth.numel())}
    if dth.numel() == 0:
        return out
    for name, d in (("theta", dth), ("phi", dph)):
        d = d.to(torch.float64)
        qs = torch.quantile(d[:: max(1, d.numel() // 1_000_000)], torch.tensor([0.5, 0.99, 0.999], dtype=torch.float64,
                                                                              device=d.device))
        out[name] = {"median": float(qs[0]), "p99": float(qs[1]), "p999": float(qs[2]), "max": float(d.max()),
                     "above_1e-6": int((d > 1e-6).sum())}
    return out


@dataclasses.dataclass(frozen=True)
class CameraRun:
    """What `timed_renders` needs of a camera workload."""
    M: float
    a: float
    term: object


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


def run_e2e_states(mb, torch, stream, flush, K: int, n: int = 1 << 20, n_steps: int = 200) -> dict:
    """End to end with inputs: the generic bound-orbit workload (n particles,
    per-particle spin, the configuration's dtau, n_steps steps), FP64.  Every
    timed step copies the initial states and spins from pinned host memory to
    the device, traces them through malbec_trace (the binding's trace), and
    copies the whole output (final states, lambda, invariants, steps, fates)
    back to pinned host memory; CUDA events on the stream bracket all three."""
    from paper_1803_08320_gb300 import workloads as W

    wl = W.bound(n=n, n_steps=n_steps)
    ics_d, spins_d, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, n, stream=stream)
    stream.synchronize()
    ics_h = torch.empty(ics_d.shape, dtype=torch.float64, pin_memory=True)
    spins_h = torch.empty(spins_d.shape, dtype=torch.float64, pin_memory=True)
    ics_h.copy_(ics_d)
    spins_h.copy_(spins_d)
    L = mb.out_layout(mb.OUT_FINAL, "fp64", n, n_steps, 0)
    out_d = torch.empty(L.total, dtype=torch.uint8, device="cuda")
    out_h = torch.empty(L.total, dtype=torch.uint8, pin_memory=True)
    times, steps = [], 0
    for k in range(K + 1):  # the first pass warms up
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            ics_d.copy_(ics_h, non_blocking=True)
            spins_d.copy_(spins_h, non_blocking=True)
            r = mb.trace(wl.M, 0.0, ics_d, wl.term, precision="fp64", a_per_ray=spins_d, stream=stream, out=out_d)
            out_h.copy_(out_d, non_blocking=True)
            e1.record(stream)
        stream.synchronize()
        if k:
            times.append(e0.elapsed_time(e1))
            steps = int(r["steps"].to(torch.int64).sum().item())
    sec = statistics.mean(times) / 1e3
    h2d = int(ics_h.numel() * 8 + spins_h.numel() * 8)
    return {"value": steps / sec, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(L.total),
            "ms_per_step": 1e3 * sec, "rk4_steps_per_step": steps,
            "workload": f"bound_orbits_{n}_a0-0.998_dtau{wl.term.dl}_{n_steps}steps_fp64",
            "note": "initial states and spins copied host->device, malbec_trace, the full output copied "
                    "device->host, every step inside the CUDA events (pinned host memory)"}


def run_workload(args) -> None:
    """--workload bundles | serving: one JSON line of its own (1 GPU)."""
    import torch

    from paper_1803_08320_gb300 import build as _b
    from paper_1803_08320_gb300 import malbec as mb

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _b.build()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    dtype = "f64" if args.precision == "fp64" else "f32+f64"
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic"}
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        if args.workload == "bundles":
            count = args.bundle_count or 4096
            # a pass of the full list takes tens of seconds: one warm-up replay
            res = run_bundles_case(mb, torch, stream, flush, count, args.precision, K=args.steps,
                                   warmup=args.warmup if count < 1024 else 1, autotune_every=max(8, count // 128),
                                   per_bundle_arm=not args.no_per_bundle_arm)
            line.update({"value": res["persistent_graph"]["value"],
                         "ms_per_step": res["persistent_graph"]["ms_per_pass"],
                         "config": {"workload": f"uneven_bundles_{count}_of_4096_size64-65536_cap1e3-1e5",
                                    "l2": res["l2"]},
                         "gpu_launches": args.steps, "bundles": res})
        elif args.workload == "paper":
            res = run_paper_case(mb, torch, stream)
            res["self_convergence"] = run_convergence_case(mb, torch, stream)
            big = res["rows"][-1]
            line.update({"value": big["final"]["steps_per_s"], "ms_per_step": 1e3 * big["final"]["seconds"],
                         "dtype": "f64",
                         "config": {"workload": "paper_sec6.4_kerr_a0.5_h0.1_1e4steps_N10-50000",
                                    "l2": "one launch per N; the inputs fit in L2 for small N"},
                         "gpu_launches": 2 * len(res["rows"]) + 1, "paper": res})
        elif args.workload == "trajectory":
            res = run_trajectory_case(mb, torch, stream, flush)
            top = [r for r in res["rows"] if r["precision"] == "fp32_mixed" and r["stride"] == 1][0]
            line.update({"value": top["steps_per_s"], "ms_per_step": 1e3 * top["seconds"], "dtype": "f32+f64",
                         "config": {"workload": "kerr_generic_bound_131072x2000_trajectory_stride1_10",
                                    "l2": "flushed before every timed launch"},
                         "gpu_launches": len(res["rows"]), "trajectory": res})
        elif args.workload == "integrators":
            res = run_integrators_case(mb, torch, stream, flush, K=args.steps, warmup=args.warmup)
            rk = res["rows"]["rk4_h0.05r"]
            line.update({"value": cw_steps_per_s(rk), "ms_per_step": rk["ms_per_render"], "dtype": "f64",
                         "config": {"workload": "kerr_camera_a0.9_1024x1024_rk4_vs_dopri5_tolerance_sweep",
                                    "l2": "flushed by a 256 MB device write before every timed render"},
                         "gpu_launches": args.steps * len(res["rows"]), "integrators": res})
        elif args.workload == "bound":
            res = run_bound_case(mb, torch, stream, flush, args.particles, args.bound_steps,
                                 ["fp64", "fp32_mixed"])
            line.update({"value": res["fp64"]["value"], "ms_per_step": 1e3 * res["fp64"]["seconds"],
                         "dtype": "f64",
                         "config": {"workload": f"kerr_generic_bound_{args.particles}x{args.bound_steps}_dtau0.02",
                                    "l2": "flushed before the timed pass; state in registers for the whole pass"},
                         "gpu_launches": 2, "bound": res})
            if "cpu_baseline" in res:
                line["cpu_baseline"] = res.pop("cpu_baseline")
        else:
            rates = [float(r) for r in args.rates.split(",")]
            res = [run_serving_case(mb, torch, rate=r, n_req=args.requests, precision=args.precision)
                   for r in rates]
            line.update({"value": statistics.mean(r["continuous_batching"]["steps_per_s"] for r in res),
                         "ms_per_step": None,
                         "config": {"workload": f"poisson_serving_{args.requests}req_per_rate",
                                    "rates": rates, "hbm_budget_bytes": 150 * 10**9},
                         "gpu_launches": sum(r["continuous_batching"]["gpu_launches"] for r in res),
                         "serving": res})
    cl = clocks.summary()
    line["clocks"] = {"sm_mhz": cl["sm_mhz"], "sm_max_mhz": cl["sm_max_mhz"], "reasons": cl["reasons"],
                      "samples": cl["samples"]}
    print(json.dumps(line))


class Ranks:
    """One process per GPU under torchrun: RANK / LOCAL_RANK / WORLD_SIZE from
    the environment; host-side barrier and max over ranks through gloo (the
    timings are host numbers; the traced rays never cross ranks)."""

    def __init__(self, world: int, rank: int, local: int):
        self.world, self.rank, self.local = world, rank, local
        if world > 1:
            import torch.distributed as dist

            dist.init_process_group("gloo")

    @classmethod
    def from_env(cls) -> "Ranks":
        return cls(int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
                   int(os.environ.get("LOCAL_RANK", "0")))

    def barrier(self) -> None:
        if self.world > 1:
            import torch.distributed as dist

            dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist

        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def close(self) -> None:
        if self.world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="malbec", choices=["malbec", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", choices=["camera_fp64", "camera_mixed", "camera_canonical", "camera_adm",
                                               "camera_dopri5", "traj_mixed", "camera_fp64_1024",
                                               "camera_mixed_1024", "camera_mixed_dopri5_1024"],
                    default=None,
                    help="case for ncu: a 512x512 render of the same camera (1024x1024 for *_1024), --steps times")
    ap.add_argument("--workload", choices=["camera", "bundles", "serving", "bound", "paper", "integrators",
                                           "trajectory"],
                    default="camera",
                    help="camera: the headline line (with a bundles and a serving sample); bundles: uneven "
                         "bundles, persistent graph launch vs one launch per bundle; serving: Poisson "
                         "arrivals at several rates, continuous batching vs one launch per request; bound: "
                         "2^20 generic bound Kerr orbits x 10^5 steps, FP64 and FP32_MIXED, drift and error "
                         "vs the oracle on a 1024-particle subsample; paper: the paper's timing experiment and "
                         "its self-convergence test; integrators: RK4 against Dormand-Prince 5(4) at several "
                         "tolerances on the camera (time, right-hand sides and invariant drift); trajectory: "
                         "strided trajectory output against the final-state mode, write bandwidth vs HBM")
    ap.add_argument("--particles", type=int, default=1 << 20, help="particles for --workload bound")
    ap.add_argument("--bound-steps", type=int, default=100_000, help="step cap for --workload bound")
    ap.add_argument("--bundle-count", type=int, default=None,
                    help="bundles taken from the 4096-bundle list (default 4096 for --workload bundles, "
                         "128 for the sample in the camera line)")
    ap.add_argument("--precision", choices=["fp64", "fp32_mixed"], default="fp32_mixed",
                    help="precision of the bundles and serving workloads")
    ap.add_argument("--rates", default="50,100,200,500,1000,2000", help="req/s for --workload serving")
    ap.add_argument("--requests", type=int, default=64, help="requests per rate for --workload serving")
    ap.add_argument("--no-extras", action="store_true", help="camera line without the bundles/serving samples")
    ap.add_argument("--no-full-configs", action="store_true",
                    help="skip the full-size generic bound-orbit and uneven-bundle runs of the default line")
    ap.add_argument("--no-per-bundle-arm", action="store_true",
                    help="--workload bundles: time the persistent graph launch only (the full 4096-bundle list "
                         "takes about ten minutes with one launch per bundle)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.workload != "camera":
        run_workload(args)
        return

    import numpy as np
    import torch

    from paper_1803_08320_gb300 import build as _b
    from paper_1803_08320_gb300 import malbec as mb

    ranks = Ranks.from_env()
    world, rank, local = ranks.world, ranks.rank, ranks.local
    torch.cuda.set_device(local)
    _b.build()
    stream = torch.cuda.Stream()
    cw, cam = camera_setup()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peak64 = mb.measure_fma_peak("fp64")
    peak32 = mb.measure_fma_peak("fp32_mixed")
    # the bare RK4 step loop of each form: the ceiling of the trace kernels
    # for their right-hand side's instruction mix
    loop = {f: mb.measure_step_loop(f) for f in (mb.FORM_GEODESIC, mb.FORM_HAMILTONIAN, mb.FORM_ADM)}

    def ceiling(form, flops_key, kernel_rate):
        fl = FLOPS_PER_STEP[flops_key]
        return {"steps_per_s": loop[form], "frac": fl * loop[form] / 1e9 / peak64,
                "kernel_over_ceiling": kernel_rate / loop[form],
                "note": "malbec_measure_step_loop: the same RK4 step with no queue, termination or output, "
                        "two warps per SM sub-partition, as the FP64 trace kernels"}
    barrier, max_over_ranks = ranks.barrier, ranks.max

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
                     "fates": fate_counts(mb, res["fate"])}
        fate64 = res["fate"].clone()
        theta64, phi64 = res["theta"].clone(), res["phi"].clone()
        t_total = max_over_ranks(sum(times64) / 1e3)
        value = world * steps_per_render * args.steps / t_total
        ms_per_step = 1e3 * t_total / args.steps

        # ---------------- FP64 and FP32_MIXED, the canonical forms (eq. Ham with
        # g of eq. kerr; with the 3+1 quantities of eq. ADM), same protocol
        def canonical_arm(form, flops_key, note):
            term_c = mb.term_from(cw.term, form=form)
            cwc = CameraRun(cw.M, cw.a, term_c)
            for _ in range(args.warmup):
                mb.trace_camera(cw.M, cw.a, cam, term_c, "fp64", stream=stream, out=out)
            barrier()
            torch.cuda.synchronize()
            times_c, res_c = timed_renders(mb, cwc, cam, "fp64", args.steps, stream, flush, out=out)
            torch.cuda.synchronize()
            barrier()
            steps_c = int(res_c["steps"].to(torch.int64).sum().item())
            t_c = max_over_ranks(sum(times_c) / 1e3)
            value_c = world * steps_c * args.steps / t_c
            agree_c = float(((res_c["fate"] & mb.FATE_MASK) == (fate64 & mb.FATE_MASK)).float().mean().item())
            esc_c = (fate64 == mb.FATE_ESCAPED) & (res_c["fate"] == mb.FATE_ESCAPED)
            dth_c = (res_c["theta"][esc_c] - theta64[esc_c]).abs()
            dph_c = (res_c["phi"][esc_c] - phi64[esc_c]).abs()
            dth_c, dph_c = dth_c[torch.isfinite(dth_c)], dph_c[torch.isfinite(dph_c)]
            fl = FLOPS_PER_STEP[flops_key]
            arm = {"value": value_c, "unit": UNIT, "ms_per_step": 1e3 * t_c / args.steps,
                   "speedup_vs_geodesic_form": value_c / value, "fate_agreement_vs_geodesic_form": agree_c,
                   "escaped_difference_vs_geodesic_form": err_stats(torch, dth_c, dph_c),
                   "roofline": {"bound": "alu", "peak": peak64, "unit": "GFLOP/s (FP64)",
                                "flops_per_rk4_step": fl,
                                "achieved": fl * steps_c / (statistics.mean(times_c) / 1e3) / 1e9,
                                "frac": fl * steps_c / (statistics.mean(times_c) / 1e3) / 1e9 / peak64},
                   "note": note}
            arm["roofline"]["step_loop_ceiling"] = ceiling(form, flops_key, value_c / world)
            fate_c, theta_c = res_c["fate"].clone(), res_c["theta"].clone()
            for _ in range(args.warmup):
                mb.trace_camera(cw.M, cw.a, cam, term_c, "fp32_mixed", stream=stream, out=out)
            barrier()
            torch.cuda.synchronize()
            times_cm, res_cm = timed_renders(mb, cwc, cam, "fp32_mixed", args.steps, stream, flush, out=out)
            torch.cuda.synchronize()
            barrier()
            steps_cm = int(res_cm["steps"].to(torch.int64).sum().item())
            t_cm = max_over_ranks(sum(times_cm) / 1e3)
            arm["fp32_mixed"] = {"value": world * steps_cm * args.steps / t_cm, "unit": UNIT,
                                 "ms_per_step": 1e3 * t_cm / args.steps,
                                 "fate_agreement_vs_fp64_same_form": float(((res_cm["fate"] & mb.FATE_MASK) ==
                                                                            (fate_c & mb.FATE_MASK)).float().mean()
                                                                           .item()),
                                 "flagged": fate_counts(mb, res_cm["fate"])["drifted_fraction"]}
            return arm, fate_c, theta_c

        canonical, fate_bl, theta_bl = canonical_arm(
            mb.FORM_HAMILTONIAN, "kerr_canonical",
            "RK4 on (x, p) with p = g u (Sec. 2, eq. Ham); same camera, inputs and outputs (x, u); "
            "the geodesic and canonical forms are different discrete maps of the same flow")
        adm_form, fate_adm, theta_adm = canonical_arm(
            mb.FORM_ADM, "kerr_adm",
            "eq. Ham with H through the lapse, shift and 3-metric of eq. ADM (Kerr's, from a provider "
            "function of r, theta); the same discrete map as the canonical form up to rounding")
        # ---------------- FP64, Dormand-Prince 5(4) with step-size control
        # (tolerance 1e-9, steps at most 0.5 r), same protocol; accuracy of
        # it and of the RK4 render against a tolerance-1e-12 reference render
        term_dp = mb.term_from(cw.term, method=mb.METHOD_DOPRI5, rtol=1e-9, atol=1e-9)
        term_dp = dataclasses.replace(term_dp, dl=0.0, dl_r_scale=0.5)
        cwd = CameraRun(cw.M, cw.a, term_dp)
        for _ in range(args.warmup):
            mb.trace_camera(cw.M, cw.a, cam, term_dp, "fp64", stream=stream, out=out)
        barrier()
        torch.cuda.synchronize()
        times_dp, res_dp = timed_renders(mb, cwd, cam, "fp64", args.steps, stream, flush, out=out)
        torch.cuda.synchronize()
        barrier()
        att_dp = int(res_dp["steps"].to(torch.int64).sum().item())
        t_dp = max_over_ranks(sum(times_dp) / 1e3)
        # accuracy: drift of the flow's invariants on 65536 of the pixels
        # (every 16th), traced as state arrays with each method
        pix = torch.arange(0, cw.n, 16, dtype=torch.int64)
        ics_s = mb.ic_camera(cw.M, cw.a, cam, pix.numpy(), stream=stream)
        drift = {}
        for name, tt in (("rk4_h0.05r", cw.term), ("dopri5_tol1e-9", term_dp)):
            rr = mb.trace(cw.M, cw.a, ics_s, tt, precision="fp64", stream=stream)
            torch.cuda.synchronize()
            ok = (rr["fate"] & mb.FATE_MASK) != mb.FATE_NONFINITE
            dd = {}
            for c, nm in enumerate(("E", "Lz", "Q", "norm")):
                d = (rr["inv1"][c] - rr["inv0"][c]).abs()[ok]
                d = d[torch.isfinite(d)]
                dd[nm] = {"median": float(d.median().item()), "p99": float(torch.quantile(d, 0.99).item())}
            drift[name] = dd
        dopri5 = {"value": world * att_dp * args.steps / t_dp, "unit": "attempts/s",
                  "ms_per_step": 1e3 * t_dp / args.steps,
                  "rays_per_s": world * cw.n * args.steps / t_dp,
                  "rays_per_s_rk4": world * cw.n * args.steps / t_total,
                  "attempts_per_ray": att_dp / cw.n, "rk4_steps_per_ray": steps_per_render / cw.n,
                  "rhs_per_ray": {"dopri5": 6.0 * att_dp / cw.n + 1.0, "rk4": 4.0 * steps_per_render / cw.n},
                  "fate_agreement_vs_rk4": float(((res_dp["fate"] & mb.FATE_MASK) == (fate64 & mb.FATE_MASK))
                                                 .float().mean().item()),
                  "flagged": fate_counts(mb, res_dp["fate"])["drifted_fraction"],
                  "roofline": {"bound": "alu", "peak": peak64, "unit": "GFLOP/s (FP64)",
                               "flops_per_attempt": FLOPS_PER_STEP["kerr_dopri5"],
                               "achieved": FLOPS_PER_STEP["kerr_dopri5"] * att_dp / (statistics.mean(times_dp) / 1e3)
                               / 1e9,
                               "frac": FLOPS_PER_STEP["kerr_dopri5"] * att_dp / (statistics.mean(times_dp) / 1e3)
                               / 1e9 / peak64},
                  "tolerance": {"rtol": 1e-9, "atol": 1e-9, "max_step": "0.5 r"},
                  "invariant_drift_65536_pixels": drift,
                  "note": "Dormand-Prince 5(4) (MALBEC_METHOD_DOPRI5), the same camera; accuracy compared by "
                          "the drift of E, L_z, Q and g(u,u) (exact invariants of the flow), since the final "
                          "angles of escaped rays depend on where each method's last step crosses r_esc"}
        # the adaptive method in FP32_MIXED (rtol >= 1e-6) against FP64 at the
        # same tolerance, same protocol
        term_dm = dataclasses.replace(term_dp, rtol=1e-6, atol=1e-6)
        cwm = CameraRun(cw.M, cw.a, term_dm)
        dm_runs = {}
        for prec in ("fp64", "fp32_mixed"):
            for _ in range(args.warmup):
                mb.trace_camera(cw.M, cw.a, cam, term_dm, prec, stream=stream, out=out)
            barrier()
            torch.cuda.synchronize()
            tt_, rr_ = timed_renders(mb, cwm, cam, prec, args.steps, stream, flush, out=out)
            torch.cuda.synchronize()
            barrier()
            rr_ = {k: v.clone() for k, v in rr_.items() if k in ("fate", "steps", "theta", "phi")}
            att_ = int(rr_["steps"].to(torch.int64).sum().item())
            t_ = max_over_ranks(sum(tt_) / 1e3)
            dm_runs[prec] = (world * att_ * args.steps / t_, 1e3 * t_ / args.steps, rr_)
        r64_, r32_ = dm_runs["fp64"][2], dm_runs["fp32_mixed"][2]
        esc_m = (r64_["fate"] == mb.FATE_ESCAPED) & (r32_["fate"] == mb.FATE_ESCAPED)
        dopri5["fp32_mixed_rtol1e-6"] = {
            "value": dm_runs["fp32_mixed"][0], "unit": "attempts/s", "ms_per_step": dm_runs["fp32_mixed"][1],
            "fp64_same_tolerance": {"value": dm_runs["fp64"][0], "ms_per_step": dm_runs["fp64"][1]},
            "speedup_vs_fp64_same_tolerance": dm_runs["fp32_mixed"][0] / dm_runs["fp64"][0],
            "fate_agreement_vs_fp64_same_tolerance": float(((r32_["fate"] & mb.FATE_MASK) == (r64_["fate"] & mb.FATE_MASK))
                                                           .float().mean().item()),
            "escaped_difference_vs_fp64_same_tolerance": err_stats(torch, (r32_["theta"][esc_m] - r64_["theta"][esc_m]).abs(),
                                                                   (r32_["phi"][esc_m] - r64_["phi"][esc_m]).abs()),
            "tolerance": {"rtol": 1e-6, "atol": 1e-6, "max_step": "0.5 r"},
            "note": "FP32 attempts on the compensated state, FP64 attempts in the FP64 zones; the difference to "
                    "FP64 at the same tolerance is of the size of the method's own error at that tolerance"}

        esc_b = (fate_bl == mb.FATE_ESCAPED) & (fate_adm == mb.FATE_ESCAPED)
        d_b = (theta_adm[esc_b] - theta_bl[esc_b]).abs()
        d_b = d_b[torch.isfinite(d_b)]
        adm_form["vs_canonical_form"] = {
            "speedup": adm_form["value"] / canonical["value"],
            "fate_agreement": float((fate_adm == fate_bl).float().mean().item()),
            "escaped_theta_difference": {"median": float(d_b.median().item()) if d_b.numel() else None,
                                         "p99": float(torch.quantile(d_b[::16], 0.99).item()) if d_b.numel()
                                         else None}}

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
        agree = float(((f32 & mb.FATE_MASK) == (fate64 & mb.FATE_MASK)).float().mean().item())
        fates32 = fate_counts(mb, f32)
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
        # end to end with input copies (states H2D, results D2H)
        e2e_states = run_e2e_states(mb, torch, stream, flush, max(1, min(args.steps, 5)))

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
                     "fp64_pipe_utilization": {
                         "pct_of_peak": load_traffic("camera_fp64", "fp64_pipe_pct_of_peak"),
                         "fp64_instructions_per_rk4_step": load_traffic("camera_fp64", "fp64_instructions_per_step"),
                         "source": "ncu sm__inst_executed_pipe_fp64 of this kernel (512x512 case, committed "
                                   "summary of the current source); the FP64-peak criterion read as pipe "
                                   "utilisation, beside the algorithmic-flop fraction above"},
                     "peak_note": "measured FP64 FMA loop on this GPU (malbec_measure_fma_peak), of measured",
                     "flops_per_rk4_step": FLOPS_PER_STEP["kerr"],
                     "plus_per_rk4_step": PLUS_PER_STEP,
                     "step_loop_ceiling": ceiling(mb.FORM_GEODESIC, "kerr", value / world)},
        "e2e": {"value": value_e2e, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(L.total),
                "note": "malbec_trace_camera + copy of the image (fate, steps, theta, phi) to pinned host memory; "
                        "the rays are built on the device from the camera description passed by value"},
        "e2e_states": e2e_states,
        "canonical_form": canonical,
        "adm_form": adm_form,
        "dopri5": dopri5,
        "fp32_mixed": {"value": value32, "unit": UNIT, "ms_per_step": 1e3 * t32 / args.steps,
                       "speedup_vs_fp64": value32 / value, "fate_agreement_vs_fp64": agree, "fates": fates32,
                       "escaped_error_vs_fp64": err_stats(torch, dth, dph),
                       "roofline": {"bound": "alu", "peak": peak32, "unit": "GFLOP/s (FP32)",
                                    "traffic": load_traffic("camera_mixed"),
                                    "issue_active_pct": load_traffic("camera_mixed", "issue_active_pct"),
                                    "achieved_fp32_equiv": FLOPS_PER_STEP["kerr"] * steps32 /
                                    (statistics.mean(times32) / 1e3) / 1e9,
                                    "frac": FLOPS_PER_STEP["kerr"] * steps32 / (statistics.mean(times32) / 1e3)
                                    / 1e9 / peak32}},
    }
    if world == 1 and not args.no_extras:
        # samples of the uneven-bundle and serving workloads (FP32_MIXED, the
        # serving default); full sweeps: --workload bundles / serving
        line["bundles_sample"] = run_bundles_case(mb, torch, stream, flush, args.bundle_count or 128,
                                                  args.precision, K=2, warmup=1)
        line["serving_sample"] = run_serving_case(mb, torch, rate=200.0, n_req=32, precision=args.precision)
        line["serving_below_saturation"] = run_serving_low_load(mb, torch, line["serving_sample"], n_req=32,
                                                                precision=args.precision)
        if not args.no_full_configs:
            # the generic bound-orbit and uneven-bundle configurations at
            # their full sizes: 2^20 orbits x 10^5 steps (FP64 and
            # FP32_MIXED, 1024-particle oracle subsample), and all 4096
            # bundles in one persistent graph launch (autotuned on every 32nd
            # bundle; the kernel is warm from the sample above)
            line["config3_bound_full"] = run_bound_case(mb, torch, stream, flush, n=1 << 20, n_steps=100_000,
                                                        precisions=("fp64", "fp32_mixed"), with_oracle=True)
            line["config4_bundles_full"] = run_bundles_case(mb, torch, stream, flush, 4096, args.precision, K=1,
                                                            warmup=0, autotune_every=32, per_bundle_arm=False,
                                                            refine_full_list=False)
        line["gpu_launches_note"] = ("gpu_launches counts the timed FP64 renders; the samples report their own "
                                     "launch counts")
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    ranks.close()


if __name__ == "__main__":
    main()

"""The request loop (malbec_server_*): host-side validation on the CPU; on
the GPU, continuous batching serves every job, each result is the same alone
and in the mix, admission respects the HBM budget and the pending limit."""
import ctypes
import math
import time

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mb():
    from paper_1803_08320_gb300 import build, malbec

    build.build()
    malbec.lib()
    return malbec


def test_server_config_validation(mb):
    lib = mb.lib()
    h = ctypes.c_void_p()
    for cfg in (mb.ServerConfig(0, 16, 16, mb.FP64, 0.01),        # no budget
                mb.ServerConfig(10**9, 0, 16, mb.FP64, 0.01),     # no active slot
                mb.ServerConfig(10**9, 5000, 16, mb.FP64, 0.01),  # too many
                mb.ServerConfig(10**9, 16, 0, mb.FP64, 0.01),
                mb.ServerConfig(10**9, 16, 16, 7, 0.01),
                mb.ServerConfig(10**9, 16, 16, mb.FP64, 0.0),
                mb.ServerConfig(10**9, 16, 16, mb.FP64, 0.01, 3, 0),          # no such form
                mb.ServerConfig(10**9, 16, 16, mb.FP32_MIXED, 0.01, 0, 2)):   # no such method
        assert lib.malbec_server_create(ctypes.byref(cfg), ctypes.byref(h)) == mb.EINVAL
    assert lib.malbec_server_destroy(None) == mb.EINVAL
    assert lib.malbec_submit(None, None, None) == mb.EINVAL


def _jobs(mb, seed=1, count=12):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        if k % 2 == 0:
            t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=2000, dl=0.0, dl_r_scale=0.05)
            cam = mb.make_camera(1000.0, math.radians(float(rng.uniform(5, 85))), 25.0, 32, 32)
            out.append(mb.make_bundle(mb.BUNDLE_CAMERA, 1024, 1.0, float(rng.uniform(0.0, 0.99)), t, camera=cam))
        else:
            t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=int(rng.integers(500, 3000)), dl=0.02)
            out.append(mb.make_bundle(mb.BUNDLE_BOUND, int(rng.integers(100, 2000)), 1.0,
                                      float(rng.uniform(0.0, 0.99)), t, seed=int(rng.integers(0, 2**62))))
    return out


def _serve(mb, jobs, precision, budget=2 * 10**9, timeout=60.0, form=0, method=0):
    import torch

    srv = mb.Server(hbm_budget=budget, max_active=64, precision=precision, idle_timeout_s=0.002, form=form,
                    method=method)
    ids = [srv.submit(b) for b in jobs]
    done, t0 = set(), time.time()
    while len(done) < len(ids):
        assert time.time() - t0 < timeout, srv.stats()
        for i in ids:
            if i not in done and srv.poll(i):
                done.add(i)
    outs = []
    for i in ids:
        o = srv.output(i)
        torch.cuda.synchronize()
        outs.append({k: v.clone() for k, v in o.items() if k not in ("buffer", "_keep")})
        srv.release(i)
    stats = srv.stats()
    srv.close()
    return outs, stats


def _same(a, b):
    import torch

    return torch.equal(torch.isnan(a), torch.isnan(b)) and torch.equal(torch.nan_to_num(a), torch.nan_to_num(b))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_results_same_alone_and_in_the_mix(mb, precision):
    jobs = _jobs(mb)
    mixed, stats = _serve(mb, jobs, precision)
    assert stats["completed"] == len(jobs) and stats["released"] == len(jobs) and stats["bytes_in_use"] == 0
    for j, b in enumerate(jobs):
        alone, _ = _serve(mb, [b], precision)
        keys = ("fate", "steps", "theta", "phi") if b.kind == mb.BUNDLE_CAMERA else ("fate", "steps", "y", "inv1")
        for k in keys:
            assert _same(mixed[j][k], alone[0][k]), (j, k)


@pytest.mark.gpu
def test_serving_matches_single_launch_fp64(mb):
    """FP64 serve results equal tracing each job alone with the bundle launch."""
    import torch

    jobs = _jobs(mb, seed=2, count=6)
    served, _ = _serve(mb, jobs, "fp64")
    for j, b in enumerate(jobs):
        (ref,) = mb.attach_outputs([b], "fp64")
        mb.trace_bundles([b], "fp64")
        torch.cuda.synchronize()
        keys = ("fate", "steps", "theta") if b.kind == mb.BUNDLE_CAMERA else ("fate", "steps", "y")
        for k in keys:
            assert _same(served[j][k], ref[k]), (j, k)


@pytest.mark.gpu
def test_admission_by_budget_and_pending_limit(mb):
    """A budget that holds one job at a time still serves them all, in
    order, as outputs are released; a full pending FIFO answers EBUSY."""
    import torch

    jobs = _jobs(mb, seed=3, count=6)
    biggest = max(mb.lib().malbec_bundle_out_bytes(ctypes.byref(b), mb.FP32_MIXED) for b in jobs)
    srv = mb.Server(hbm_budget=biggest, max_active=64, max_pending=3, precision="fp32_mixed", idle_timeout_s=0.002)
    ids = [srv.try_submit(b) for b in jobs]
    # one admitted (budget), three pending, the rest refused
    assert all(i is not None for i in ids[:4]) and ids[4] is None and ids[5] is None
    st = srv.stats()
    assert st["active"] + st["completed"] <= 1 and st["pending"] == 3
    served, t0 = [], time.time()
    while len(served) < 4:
        assert time.time() - t0 < 60, srv.stats()
        for i in ids[:4]:
            if i not in served and srv.poll(i):
                srv.output(i)
                torch.cuda.synchronize()
                srv.release(i)
                served.append(i)
    assert served == ids[:4]  # FIFO admission with a one-job budget
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def _in_class(mb, jobs, form, method, tol=1e-9):
    """The same jobs in another class (form, method); Dormand-Prince at
    tolerance `tol`."""
    for b in jobs:
        t = mb.Termination(b.term.eps_hor, b.term.r_esc, b.term.n_steps_cap, b.term.dl, b.term.dl_r_scale, form,
                           method, tol if method else 0.0, tol if method else 0.0)
        b.term = t.c()
    return jobs


@pytest.mark.gpu
@pytest.mark.parametrize("precision,form,method", [("fp32_mixed", 1, 0), ("fp32_mixed", 2, 0), ("fp64", 2, 0),
                                                   ("fp64", 0, 1), ("fp64", 1, 1), ("fp32_mixed", 0, 1),
                                                   ("fp32_mixed", 2, 1)])
def test_server_of_another_class_alone_and_in_the_mix(mb, precision, form, method):
    """A server runs one class of jobs (form, method): the canonical forms
    (eq. Ham through eq. kerr and eq. ADM) and Dormand-Prince (FP64 at 1e-9,
    FP32_MIXED at 1e-6) are served with the same guarantees -- each result
    bitwise the same alone and in the mix, FP64 and FP32_MIXED
    Dormand-Prince results equal to tracing the job alone with the bundle
    launch (no block exchange in either) -- and a job of another class, or
    (FP32_MIXED Dormand-Prince) below the tolerance floor, is refused."""
    import torch

    tol = 1e-6 if (precision == "fp32_mixed" and method == 1) else 1e-9
    jobs = _in_class(mb, _jobs(mb, seed=4, count=6), form, method, tol)
    mixed, stats = _serve(mb, jobs, precision, form=form, method=method)
    assert stats["completed"] == len(jobs)
    for j, b in enumerate(jobs):
        alone, _ = _serve(mb, [b], precision, form=form, method=method)
        keys = ("fate", "steps", "theta", "phi") if b.kind == mb.BUNDLE_CAMERA else ("fate", "steps", "y", "inv1")
        for k in keys:
            assert _same(mixed[j][k], alone[0][k]), (j, k)
        if precision == "fp64" or method == 1:
            (ref,) = mb.attach_outputs([b], precision)
            mb.trace_bundles([b], precision)
            torch.cuda.synchronize()
            for k in keys:
                assert _same(mixed[j][k], ref[k]), (j, k)
    srv = mb.Server(hbm_budget=10**9, precision=precision, form=form, method=method)
    other = _jobs(mb, seed=9, count=1)[0]  # geodesic RK4
    if (form, method) != (0, 0):
        with pytest.raises(mb.MalbecError):
            srv.submit(other)
    if precision == "fp32_mixed" and method == 1:
        (below_floor,) = _in_class(mb, _jobs(mb, seed=9, count=1), form, method, 0.5e-6)
        with pytest.raises(mb.MalbecError):
            srv.submit(below_floor)
    srv.close()


@pytest.mark.gpu
def test_canonical_server_job_matches_oracle(mb, orc):
    """A BOUND job on an FP64 server of the canonical form through eq. ADM:
    states within 1e-9 of the oracle's form 2."""
    import torch

    from test_gpu_parity import RTOL, assert_states_close, oracle_term

    a, seed, n = 0.6, 4242, 48
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=500, dl=0.02, form=2)
    b = mb.make_bundle(mb.BUNDLE_BOUND, n, 1.0, a, t, seed=seed)
    (out,), _ = _serve(mb, [b], "fp64", form=2)
    torch.cuda.synchronize()
    ys, _, _ = orc.bound_samples(1.0, a, seed, np.arange(n), spin_fixed=True)
    ref = orc.trace_many(1.0, a, ys, oracle_term(orc, t))
    assert np.array_equal(out["fate"].cpu().numpy(), ref["fate"])
    assert_states_close(out["y"].cpu().numpy(), ref["y"], rtol=RTOL)

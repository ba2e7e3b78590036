"""The Dormand-Prince 5(4) integrator with step-size control
(MALBEC_METHOD_DOPRI5, FP64) on the GPU against the oracle's method 1 in
each form (the geodesic equation, and the canonical equations through
g^{mu nu} of eq. kerr or the 3+1 quantities of eq. ADM): the same tableau,
error norm and controller, so the same sequence of attempts up to rounding.
States within 1e-9 per component, attempt counts and fates equal, on the rays
whose oracle map is insensitive to rounding (bound orbits: measured with the
oracle's rhs_noise option) or well conditioned (cameras and samples: kappa).
"""
import dataclasses

import numpy as np
import pytest

from test_gpu_parity import (KAPPA_MAX, _camera_compare, assert_states_close, gpu_trace, np_, oracle_kappa,
                             oracle_term)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    import torch

    from paper_1803_08320_gb300 import build, malbec

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    malbec.lib()
    return malbec


@pytest.fixture(scope="module")
def W():
    from paper_1803_08320_gb300 import workloads

    return workloads


@pytest.fixture(scope="module", params=[0, 1, 2], ids=["geodesic", "kerr_bl", "adm"])
def form(request):
    return request.param


def dp_term(mb, tol=1e-10, **kw):
    base = dict(eps_hor=0.01, r_esc=1100.0, n_steps_cap=3000, dl=0.02, method=mb.METHOD_DOPRI5, rtol=tol, atol=tol)
    base.update(kw)
    return mb.Termination(**base)


SENS_MAX = 1e-10


def oracle_rounding_sensitivity(orc, M, a, ics, t_or, a_per_ray=None):
    """Per ray, how far the oracle's own result moves when every component of
    every right-hand-side evaluation is perturbed by +-1 unit in the last
    place (the oracle's rhs_noise option, two sign patterns: delta = 2^-52
    and 1.5 x 2^-52): the largest relative change of the final state, +inf
    where the number of attempts, lambda or the fate changed.  Two correct
    FP64 implementations of the adaptive map differ by rounding of about that
    size on every evaluation, so a ray whose result moves by more than
    SENS_MAX cannot be compared at 1e-9: its adaptive map sits at a step
    decision the rounding can flip, or amplifies rounding (passages next to
    the polar axis)."""
    ref = orc.trace_many(M, a, ics, t_or, a_per_ray=a_per_ray)
    sens = np.zeros(ics.shape[1])
    for delta in (2.0**-52, 1.5 * 2.0**-52):
        t1 = orc.make_term(t_or.eps_hor, t_or.r_esc, t_or.n_steps_cap, t_or.dl, t_or.dl_r_scale, t_or.form,
                           t_or.method, t_or.rtol, t_or.atol, delta)
        per = orc.trace_many(M, a, ics, t1, a_per_ray=a_per_ray)
        with np.errstate(invalid="ignore"):
            rel = (np.abs(per["y"] - ref["y"]) / np.maximum(np.abs(ref["y"]), 1.0)).max(axis=0)
        rel = np.where(np.isfinite(rel), rel, np.inf)
        moved = (per["steps"] != ref["steps"]) | (per["lambda"] != ref["lambda"]) | (per["fate"] != ref["fate"])
        sens = np.maximum(sens, np.where(moved, np.inf, rel))
    return ref, sens


def test_bound_orbits_match_oracle(mb, orc, W, form):
    """512 generic bound orbits (per-particle spin), 3000 attempts at
    tolerance 1e-10.  The adaptive map is discontinuous where an attempt's
    error norm sits at the acceptance threshold or carries a step exponent
    across an integer, and a step across a near-polar passage amplifies the
    rounding of each stage; the oracle's own rounding sensitivity (above)
    finds those rays.  On every other orbit (at least 95%; measured 97-98%)
    the GPU takes the oracle's sequence of attempts (count and lambda equal,
    bit for bit), ends with its fate, and every state component is within
    1e-9.  Every capped orbit, the excluded ones included, keeps E, L_z, Q
    and the norm within 3000 x tol of their initial values."""
    wl = W.bound()
    idx = wl.subsample(512)
    ys, spins, _ = orc.bound_samples(wl.M, wl.a_max, wl.seed, idx)
    t = dp_term(mb, form=form)
    got = gpu_trace(mb, wl.M, 0.0, ys, t, a_per_ray=spins)
    ref, sens = oracle_rounding_sensitivity(orc, wl.M, 0.0, ys, oracle_term(orc, t), a_per_ray=spins)
    good = sens <= SENS_MAX
    print("form", form, "rounding-sensitive orbits excluded:", int((~good).sum()), "of", len(good))
    assert good.mean() >= 0.95, good.mean()
    # with a fixed first step and no r-proportional cap every step is
    # dl 2^(m/4): the same sequence of steps gives the same lambda, bit for bit
    assert np.array_equal(got["steps"][good].astype(np.uint32), ref["steps"][good])
    assert np.array_equal(got["lambda"][good], ref["lambda"][good])
    assert np.array_equal(got["fate"][good], ref["fate"][good])
    assert_states_close(got["y"][:, good], ref["y"][:, good], what="Dormand-Prince bound orbits")
    capped = (got["fate"] & mb.FATE_MASK) == mb.FATE_CAPPED
    assert capped.mean() > 0.95
    drift = np.abs(got["inv1"][:, capped] - got["inv0"][:, capped]) / np.maximum(np.abs(got["inv0"][:, capped]), 1.0)
    assert drift.max() <= 3000 * 1e-10, drift.max(axis=1)


def test_circular_orbits_and_step_growth(mb, W):
    """Schwarzschild circular orbits from a tiny first step (1e-4): the
    controller grows it by orders of magnitude and r stays at r0.  (An exact
    circular orbit has no truncation error -- (r, theta, u) is a fixed point
    of the right-hand side -- so its error estimate is rounding noise alone
    and its sequence of steps is not compared with the oracle's.)"""
    wl = W.circular(n=128)
    ics = np_(mb.ic_circular(1.0, 0.0, wl.radii))
    t = dp_term(mb, tol=1e-11, dl=1e-4, n_steps_cap=2000)
    got = gpu_trace(mb, 1.0, 0.0, ics, t)
    assert (got["fate"] == mb.FATE_CAPPED).all()
    assert np.abs(got["y"][1] - wl.radii).max() < 1e-6
    assert got["lambda"].min() > 100 * 1e-4 * 2000
    d = np.abs(got["inv1"][:2] - got["inv0"][:2]) / np.abs(got["inv0"][:2])
    assert d.max() < 1e-9


def test_camera_small_image(mb, orc, W, form):
    """48 x 48 Kerr a = 0.9 camera with the adaptive integrator (tolerance
    1e-9, steps at most 0.5 r): fates and attempt counts of well-conditioned
    pixels away from the critical curve equal the oracle's; escaped (theta,
    phi) within 1e-9."""
    import torch

    cw = W.camera(nx=48, ny=48)
    cw = dataclasses.replace(cw, term=dp_term(mb, tol=1e-9, dl=0.0, dl_r_scale=0.5, n_steps_cap=20_000, form=form))
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    res = mb.trace_camera(cw.M, cw.a, cam, cw.term, "fp64")
    torch.cuda.synchronize()
    got = {k: np_(v) for k, v in res.items() if k != "buffer"}
    pix = np.arange(cw.n)
    ref, near, agree, far = _camera_compare(mb, orc, cw, got, pix, form=form)
    good = ref["kappa"] <= KAPPA_MAX
    assert agree[far & good].all()
    assert np.array_equal(got["steps"][far & good].astype(np.uint32), ref["steps"][far & good])
    esc = far & good & (ref["fate"] == mb.FATE_ESCAPED)
    assert esc.sum() > 500
    assert_states_close(got["theta"][esc], ref["y"][2][esc], what="theta")
    assert_states_close(got["phi"][esc], ref["y"][3][esc], what="phi")


def test_strided_samples(mb, orc, form):
    """Samples every `stride` attempts (a rejected attempt repeats the last
    accepted state) of eccentric orbits (circular ones with u^r = 0.01) equal
    the oracle's within 1e-9 where the sequence of steps is the oracle's;
    NaN after the end."""
    rng = np.random.default_rng(5)
    ys = np.stack([orc.circular_state(1.0, 0.5, r, 1) for r in rng.uniform(7.0, 12.0, 24)], axis=1)
    ys[5] = 0.01
    t = dp_term(mb, tol=1e-9, r_esc=40.0, n_steps_cap=600, dl=0.5, form=form)
    got = gpu_trace(mb, 1.0, 0.5, ys, t, mode=mb.OUT_STRIDED, stride=25)
    ref = orc.trace_many(1.0, 0.5, ys, oracle_term(orc, t), stride=25, want_traj=True)
    same = (got["steps"].astype(np.uint32) == ref["steps"]) & (got["lambda"] == ref["lambda"])
    assert same.mean() >= 0.9, same.mean()
    assert np.array_equal(np.isnan(got["traj"][same]), np.isnan(ref["traj"][same]))
    fin = ~np.isnan(ref["traj"][same])
    assert_states_close(got["traj"][same][fin], ref["traj"][same][fin], what="Dormand-Prince samples")


def test_more_accurate_than_rk4_on_camera_rays(mb, W):
    """4096 rays of the camera workload traced as state arrays: with the
    camera's step rule RK4 and the adaptive method at tolerance 1e-9 (steps
    at most 0.5 r) agree on >= 99% of the fates, and the adaptive method
    keeps the Carter constant and the null norm, exact invariants of the
    flow, closer to their initial values."""
    import torch

    cw = W.camera(nx=64, ny=64)
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    ics = mb.ic_camera(cw.M, cw.a, cam, np.arange(cw.n))
    rk = mb.trace(cw.M, cw.a, ics, cw.term)
    dp = mb.trace(cw.M, cw.a, ics, dp_term(mb, tol=1e-9, dl=0.0, dl_r_scale=0.5, n_steps_cap=20_000))
    torch.cuda.synchronize()
    m = mb.FATE_MASK
    assert ((dp["fate"] & m) == (rk["fate"] & m)).float().mean().item() >= 0.99

    def drift(r, c):
        ok = (r["fate"] & m) != mb.FATE_NONFINITE
        d = (r["inv1"][c] - r["inv0"][c]).abs()[ok]
        return d[torch.isfinite(d)].median().item()

    assert drift(dp, 2) < drift(rk, 2)   # Q
    assert drift(dp, 3) < drift(rk, 3)   # g(u, u)


def test_unsupported_combinations_are_rejected(mb):
    ics = np.zeros((8, 4))
    ics[1] = 10.0
    ics[2] = 1.0
    ics[4] = 1.2
    # FP32_MIXED takes the adaptive method at rtol >= MALBEC_DOPRI5_MIXED_RTOL_MIN only
    with pytest.raises(mb.MalbecError):
        gpu_trace(mb, 1.0, 0.5, ics, dp_term(mb), precision="fp32_mixed")
    with pytest.raises(mb.MalbecError):
        gpu_trace(mb, 1.0, 0.5, ics, dp_term(mb, tol=0.5e-6), precision="fp32_mixed")
    assert gpu_trace(mb, 1.0, 0.5, ics, dp_term(mb, tol=1e-6, n_steps_cap=50), precision="fp32_mixed")["fate"].size == 4
    # job tables: the same floor
    b = mb.make_bundle(mb.BUNDLE_BOUND, 4, 1.0, 0.5, dp_term(mb, tol=0.5e-6), seed=1)
    with pytest.raises(mb.MalbecError):
        mb.attach_outputs([b], "fp32_mixed")
        mb.trace_bundles([b], "fp32_mixed")


def test_noalloc_entry_point_gives_the_same_bits(mb, W):
    """The adaptive integrator through malbec_trace_noalloc: the same kernel
    as malbec_trace, so the same bits; FP32_MIXED is rejected there too."""
    import torch

    wl = W.bound()
    ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, 300)
    t = dp_term(mb, n_steps_cap=500)
    a = mb.trace(wl.M, 0.0, ics, t, a_per_ray=spins)
    L = mb.out_layout(mb.OUT_FINAL, "fp64", 300, t.n_steps_cap, 0)
    out = torch.empty(L.total, dtype=torch.uint8, device="cuda")
    b = mb.trace_noalloc(wl.M, 0.0, ics, t, out, a_per_ray=spins)
    torch.cuda.synchronize()
    for k in ("y", "lambda", "steps", "fate", "inv1"):
        assert torch.equal(a[k], b[k]), k
    with pytest.raises(mb.MalbecError):
        mb.trace_noalloc(wl.M, 0.0, ics, t, out, precision="fp32_mixed", a_per_ray=spins)
    with pytest.raises(mb.MalbecError):
        mb.trace_noalloc(wl.M, 0.0, ics, dp_term(mb, tol=1e-6, n_steps_cap=500), out, precision="fp32_mixed",
                         a_per_ray=spins)


def test_every_form_conserves_the_invariants(mb, W):
    """With the adaptive integrator at tolerance 1e-11 every form keeps the
    flow's invariants: Q and the norm within 1500 x tol after 1500 attempts
    on >= 95% of the bound-orbit sample, and in the canonical forms E and L_z
    to the rounding of the conversions at the two ends.  (The forms take
    different step sequences, so their end states sit at different lambda.)"""
    import torch

    wl = W.bound()
    ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, 1024)
    for f in (0, 1, 2):
        r = mb.trace(wl.M, 0.0, ics, dp_term(mb, tol=1e-11, n_steps_cap=1500, form=f), a_per_ray=spins)
        torch.cuda.synchronize()
        ok = r["fate"] == mb.FATE_CAPPED
        assert ok.float().mean().item() > 0.95
        d = (r["inv1"][:, ok] - r["inv0"][:, ok]).abs() / r["inv0"][:, ok].abs().clamp(min=1.0)
        assert (d[2:].amax(dim=0) <= 1500 * 1e-11).float().mean().item() >= 0.95, f
        if f != 0:
            assert d[:2].max().item() < 1e-12, f


# --------------------------------------------------------------------------- FP32_MIXED
def test_mixed_camera_against_the_oracle(mb, orc, W, form):
    """The adaptive method in FP32_MIXED (FP32 attempts on the compensated
    state, FP64 attempts in the FP64 zones) at rtol = atol = 1e-6 on a 48 x 48
    Kerr a = 0.9 camera, against the oracle's method 1 at the same tolerance
    and against the oracle at 1e-11.  Away from the critical curve and the
    polar axis: terminations equal the oracle's on >= 99.9% of the pixels
    (measured 100%); the escaped angles equal the oracle's to a median of
    1e-6 (measured 6e-8: most rays take the oracle's sequence of attempts);
    and against the 1e-11 render the FP32_MIXED error is the method's own at
    this tolerance -- its p99 within 1.2x the oracle's own p99 at 1e-6 (both
    measured 3.7e-3 to 6.0e-3)."""
    import math

    import torch

    from test_gpu_parity import _camera_near, _pixel_ab, sin_theta_turn

    cw = W.camera(nx=48, ny=48)
    t = dp_term(mb, tol=1e-6, dl=0.0, dl_r_scale=0.5, n_steps_cap=20_000, form=form)
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    res = mb.trace_camera(cw.M, cw.a, cam, t, "fp32_mixed")
    torch.cuda.synchronize()
    got = {k: np_(v) for k, v in res.items() if k != "buffer"}
    pix = np.arange(cw.n)
    ics = orc.camera_ics(cw.M, cw.a, cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny, pix)
    ref = orc.trace_many(cw.M, cw.a, ics, oracle_term(orc, t))
    tight = orc.trace_many(cw.M, cw.a, ics, oracle_term(orc, dp_term(mb, tol=1e-11, dl=0.0, dl_r_scale=0.5,
                                                                        n_steps_cap=20_000, form=form)))
    al, be = _pixel_ab(cw, pix)
    Lz = -al * math.sin(cw.incl)
    Q = be * be + math.cos(cw.incl) ** 2 * (al * al - cw.a * cw.a)
    sel = ~_camera_near(orc, cw, pix) & (sin_theta_turn(1.0, Lz, Q, cw.a, 0.0) >= 0.05)
    m = mb.FATE_MASK
    same = (got["fate"] & m) == (ref["fate"] & m)
    esc = sel & (got["fate"] == mb.FATE_ESCAPED) & (ref["fate"] == mb.FATE_ESCAPED) & \
        (tight["fate"] == mb.FATE_ESCAPED)
    e_same = np.abs(got["theta"][esc] - ref["y"][2][esc])
    e_mixed = np.abs(got["theta"][esc] - tight["y"][2][esc])
    e_oracle = np.abs(ref["y"][2][esc] - tight["y"][2][esc])
    print("form", form, "fates", same[sel].mean(), "escaped", esc.sum(), "theta vs same tol median",
          np.median(e_same), "p99 vs 1e-11: mixed", np.quantile(e_mixed, 0.99), "oracle", np.quantile(e_oracle, 0.99))
    assert sel.sum() > 1000 and esc.sum() > 600
    assert same[sel].mean() >= 0.999
    assert np.median(e_same) <= 1e-6
    assert np.quantile(e_mixed, 0.99) <= 1.2 * np.quantile(e_oracle, 0.99)


def test_mixed_bound_orbits_keep_the_invariants_as_fp64(mb, orc, W, form):
    """512 generic bound orbits, 3000 attempts at rtol = atol = 1e-6: the
    FP32_MIXED adaptive method drifts from E, L_z, Q and g(u,u) as the FP64
    one does at the same tolerance (median and p99 of each within 1.5x of
    FP64's, measured within 5%: the error is the method's, not FP32
    rounding's), and in the canonical forms E and L_z stay exact to the
    conversions at the two ends (<= 1e-13)."""
    wl = W.bound()
    idx = wl.subsample(512)
    ys, spins, _ = orc.bound_samples(wl.M, wl.a_max, wl.seed, idx)
    t = dp_term(mb, tol=1e-6, n_steps_cap=3000, form=form)
    runs = {p: gpu_trace(mb, wl.M, 0.0, ys, t, a_per_ray=spins, precision=p) for p in ("fp64", "fp32_mixed")}
    capped = np.ones(ys.shape[1], dtype=bool)
    for r in runs.values():
        capped &= (r["fate"] & mb.FATE_MASK) == mb.FATE_CAPPED
    assert capped.mean() > 0.95

    def drift(r):
        return np.abs(r["inv1"][:, capped] - r["inv0"][:, capped]) / np.maximum(np.abs(r["inv0"][:, capped]), 1.0)

    d64, d32 = drift(runs["fp64"]), drift(runs["fp32_mixed"])
    for c in (2, 3) if form != 0 else (0, 1, 2, 3):
        for qq in (0.5, 0.99):
            assert np.quantile(d32[c], qq) <= 1.5 * np.quantile(d64[c], qq) + 1e-12, (c, qq)
    if form != 0:
        assert d32[:2].max() <= 1e-13




def test_mixed_strided_samples(mb, orc):
    """FP32_MIXED adaptive samples every 25 attempts of eccentric orbits
    (circular ones with u^r = 0.01 and u^theta = 0.004, so Q > 0; one
    starting inside the capture radius)
    at rtol = atol = 1e-6: FP32 samples (the state's hi words), sample 0 the
    initial state rounded to FP32, sample k finite exactly when k x 25 <= the
    attempts taken (NaN after the end), and a capped orbit's last sample its
    final state to one FP32 unit.  The step sequences part from the oracle's
    (FP64, same tolerance) after a few hundred attempts, so the samples are
    checked on the flow's invariants: the largest change of E, L_z, Q and
    g(u,u) over a ray's samples stays within 1.5x the oracle's own over its
    samples (median and p90 over the rays; measured within 10%) plus the
    FP32 rounding of a sample (1e-6)."""
    rng = np.random.default_rng(5)
    ys = np.stack([orc.circular_state(1.0, 0.5, r, 1) for r in rng.uniform(7.0, 12.0, 24)], axis=1)
    ys[5], ys[6] = 0.01, 0.004
    ys[1, 0] = 1.87  # inside the capture radius (1.01 r+ = 1.885), outside r+: ends at its first attempt
    t = dp_term(mb, tol=1e-6, r_esc=40.0, n_steps_cap=600, dl=0.5)
    got = gpu_trace(mb, 1.0, 0.5, ys, t, mode=mb.OUT_STRIDED, stride=25, precision="fp32_mixed")
    ref = orc.trace_many(1.0, 0.5, ys, oracle_term(orc, t), stride=25, want_traj=True)
    traj = got["traj"]
    n, ns = ys.shape[1], 600 // 25 + 1
    assert traj.shape == (n, ns, 8) and traj.dtype == np.float32
    assert np.array_equal(traj[:, 0, :], ys.T.astype(np.float32))
    steps = got["steps"].astype(np.int64)
    want_fin = np.arange(ns)[None, :] * 25 <= steps[:, None]
    assert np.array_equal(np.isfinite(traj).all(axis=2), want_fin)
    assert np.array_equal(np.isnan(traj).all(axis=2), ~want_fin)
    capped = (got["fate"] & mb.FATE_MASK) == mb.FATE_CAPPED
    assert capped.sum() >= 20 and got["fate"][0] == mb.FATE_CAPTURED
    assert np.array_equal(got["fate"], ref["fate"])
    y_end = got["y"][:, capped].T
    assert (np.abs(traj[capped, -1, :] - y_end) <= np.spacing(np.abs(y_end).astype(np.float32))).all()

    def inv_drift(tr):
        out = np.zeros((4, int(capped.sum())))
        for j, i in enumerate(np.flatnonzero(capped)):
            inv = np.stack([orc.invariants(1.0, 0.5, tr[i, k].astype(np.float64)) for k in range(ns)], axis=1)
            out[:, j] = (np.abs(inv - inv[:, :1]) / np.maximum(np.abs(inv[:, :1]), 1.0)).max(axis=1)
        return out

    d32, d64 = inv_drift(traj), inv_drift(ref["traj"])
    for c in range(4):
        for qq in (0.5, 0.9):
            print("invariant", c, "q", qq, "mixed", np.quantile(d32[c], qq), "oracle", np.quantile(d64[c], qq))
            assert np.quantile(d32[c], qq) <= 1.5 * np.quantile(d64[c], qq) + 1e-6, (c, qq)

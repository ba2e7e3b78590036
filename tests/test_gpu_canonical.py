"""The canonical form (Sec. 2, eq. Ham: RK4 on (x^mu, p_mu) with p = g u) on
the GPU against the oracle's canonical trace, with the tolerance of the
geodesic form (1e-9 per component, reading G11): circular orbits, generic
bound orbits, the camera, strided trajectories; and p_t, p_phi exactly
constant."""
import dataclasses
import math

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


def canonical(mb, t):
    return mb.Termination(t.eps_hor, t.r_esc, t.n_steps_cap, t.dl, t.dl_r_scale, mb.FORM_HAMILTONIAN)


def test_circular_orbits(mb, orc, W):
    """Schwarzschild (the Kerr Hamiltonian at a = 0) and Kerr a = 0.7
    circular orbits, 10^4 steps of 0.01: within 1e-9 of the oracle; r stays
    at r0; E and L_z unchanged to the conversion round trip."""
    wl = W.circular()
    for a, radii in ((0.0, wl.radii), (0.7, wl.radii[:256] + 2.0)):
        ics = np_(mb.ic_circular(1.0, a, radii))
        t = canonical(mb, wl.term)
        got = gpu_trace(mb, 1.0, a, ics, t)
        ref = orc.trace_many(1.0, a, ics, oracle_term(orc, t))
        assert_states_close(got["y"], ref["y"], what=f"canonical circular a={a}")
        assert np.array_equal(got["steps"].astype(np.uint32), ref["steps"])
        assert np.abs(got["y"][1] - radii).max() < 1e-9 * 22
        d = np.abs(got["inv1"][:2] - got["inv0"][:2]) / np.abs(got["inv0"][:2])
        assert d.max() < 1e-13


def test_bound_orbits_subsample(mb, orc, W):
    """The generic bound-orbit subsample (1024 particles, 10^4 steps of 0.02,
    per-particle spin) within 1e-9 of the oracle's canonical trace, apart from
    the few orbits whose discrete map is ill-conditioned next to the polar
    axis (reading G19); E and L_z conserved to 1e-12."""
    wl = W.bound()
    idx = wl.subsample(1024)
    ys, spins, _ = orc.bound_samples(wl.M, wl.a_max, wl.seed, idx)
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=10_000, dl=0.02, form=mb.FORM_HAMILTONIAN)
    got = gpu_trace(mb, wl.M, 0.0, ys, t, a_per_ray=spins)
    ref, kappa = oracle_kappa(orc, wl.M, 0.0, ys, oracle_term(orc, t), a_per_ray=spins)
    good = kappa <= KAPPA_MAX
    assert (~good).mean() <= 0.01
    assert np.array_equal(got["fate"][good], ref["fate"][good])
    assert np.array_equal(got["steps"][good].astype(np.uint32), ref["steps"][good])
    assert_states_close(got["y"][:, good], ref["y"][:, good], what="canonical bound orbits")
    capped = good & (got["fate"] == mb.FATE_CAPPED)
    d = np.abs(got["inv1"][:2, capped] - got["inv0"][:2, capped]) / np.maximum(np.abs(got["inv0"][:2, capped]), 1.0)
    assert d.max() < 1e-12


def test_camera_small_image(mb, orc, W):
    """64 x 64 Kerr a = 0.9 camera in the canonical form: fates and steps of
    well-conditioned pixels away from the critical curve equal the oracle's;
    escaped (theta, phi) within 1e-9."""
    import torch

    cw = W.camera(nx=64, ny=64)
    cw = dataclasses.replace(cw, term=canonical(mb, cw.term))
    cam = mb.make_camera(cw.r_obs, cw.incl, cw.fov_half, cw.nx, cw.ny)
    res = mb.trace_camera(cw.M, cw.a, cam, cw.term, "fp64")
    torch.cuda.synchronize()
    got = {k: np_(v) for k, v in res.items() if k != "buffer"}
    pix = np.arange(cw.n)
    ref, near, agree, far = _camera_compare(mb, orc, cw, got, pix, form=1)
    good = ref["kappa"] <= KAPPA_MAX
    assert agree[far & good].all()
    assert agree[far].mean() >= 0.9999
    assert np.array_equal(got["steps"][far & good].astype(np.uint32), ref["steps"][far & good])
    esc = far & good & (ref["fate"] == mb.FATE_ESCAPED)
    assert esc.sum() > 1000
    assert_states_close(got["theta"][esc], ref["y"][2][esc], what="theta")
    assert_states_close(got["phi"][esc], ref["y"][3][esc], what="phi")


def test_strided_trajectories(mb, orc):
    """Trajectory samples of the canonical form are (x, u) states equal to the
    oracle's samples within 1e-9; samples after termination are NaN."""
    rng = np.random.default_rng(4)
    ys = np.stack([orc.circular_state(1.0, 0.5, r, 1) for r in rng.uniform(7.0, 12.0, 20)], axis=1)
    ys[5] *= 1.0 + 0.02 * rng.standard_normal(ys.shape[1])
    t = mb.Termination(eps_hor=0.01, r_esc=60.0, n_steps_cap=800, dl=0.05, form=mb.FORM_HAMILTONIAN)
    got = gpu_trace(mb, 1.0, 0.5, ys, t, mode=mb.OUT_STRIDED, stride=50)
    ref = orc.trace_many(1.0, 0.5, ys, oracle_term(orc, t), stride=50, want_traj=True)
    tg, tr = got["traj"], ref["traj"]
    assert np.array_equal(np.isnan(tg), np.isnan(tr))
    fin = ~np.isnan(tr)
    assert_states_close(tg[fin], tr[fin], what="canonical trajectory samples")


def test_canonical_agrees_with_geodesic_form(mb, W):
    """The two forms integrate the same flow: on smooth orbits their results
    differ by the RK4 truncation error only (well below 1e-6 here)."""
    ics = np_(mb.ic_bound(1.0, 0.5, W.bound().seed, 256, spin_fixed=True)[0])
    t0 = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=2000, dl=0.02)
    g = gpu_trace(mb, 1.0, 0.5, ics, t0)
    c = gpu_trace(mb, 1.0, 0.5, ics, dataclasses.replace(t0, form=mb.FORM_HAMILTONIAN))
    ok = (g["fate"] == mb.FATE_CAPPED) & (c["fate"] == mb.FATE_CAPPED)
    assert ok.mean() > 0.95
    rel = np.abs(g["y"][:, ok] - c["y"][:, ok]) / np.maximum(np.abs(g["y"][:, ok]), 1.0)
    assert np.median(rel.max(axis=0)) < 1e-7


def test_canonical_rejects_mixed_and_job_tables(mb):
    import torch

    t = mb.Termination(eps_hor=0.01, r_esc=60.0, n_steps_cap=10, dl=0.05, form=mb.FORM_HAMILTONIAN)
    ics = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    ics[1] = 10.0
    ics[2] = math.pi / 2
    with pytest.raises(mb.MalbecError):
        mb.trace(1.0, 0.5, ics, t, precision="fp32_mixed")
    b = mb.make_bundle(mb.BUNDLE_BOUND, 4, 1.0, 0.5, t, seed=1)
    with pytest.raises(mb.MalbecError):
        mb.attach_outputs([b], "fp64")
        mb.trace_bundles([b], "fp64")

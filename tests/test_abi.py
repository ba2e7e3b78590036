"""The C-ABI library builds, loads and exports every entry point that
include/malbec.h declares; host-only logic (layouts, argument validation that
rejects before any CUDA call) is checked without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "malbec.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(malbec_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def mb():
    from paper_1803_08320_gb300 import build, malbec

    build.build()
    return malbec


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("malbec_trace", "malbec_trace_camera", "malbec_out_layout", "malbec_ic_circular",
                 "malbec_ic_bound", "malbec_invariants", "malbec_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(mb):
    lib = mb.lib()
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_build_info(mb):
    assert mb.strerror(0) == "ok"
    assert "invalid" in mb.strerror(-1)
    assert mb.strerror(-99) == "unknown error code"
    assert "sm_103a" in mb.build_info()


def test_out_layout_alignment_and_sizes(mb):
    n, cap, stride = 1000, 1000, 10
    L = mb.out_layout(mb.OUT_STRIDED, "fp64", n, cap, stride)
    offs = [L.y, L.lam, L.inv0, L.inv1, L.steps, L.fate, L.traj]
    assert all(o % 256 == 0 for o in offs)
    assert offs == sorted(offs)
    assert L.lam >= L.y + 8 * n * 8 and L.inv0 >= L.lam + 8 * n
    assert L.steps >= L.inv1 + 32 * n and L.fate >= L.steps + 4 * n
    assert L.n_samples == cap // stride + 1
    assert L.total >= L.traj + n * L.n_samples * 64
    L32 = mb.out_layout(mb.OUT_STRIDED, "fp32_mixed", n, cap, stride)
    assert L32.total - L32.traj == pytest.approx((L.total - L.traj) / 2, abs=256)
    Lf = mb.out_layout(mb.OUT_FINAL, "fp64", n, cap, 0)
    assert Lf.traj == 0 and Lf.n_samples == 0
    assert mb.lib().malbec_out_bytes(mb.OUT_FINAL, mb.FP64, n, cap, 0) == Lf.total


def test_out_layout_rejects_bad_arguments(mb):
    lib = mb.lib()
    L = mb.Layout()
    assert lib.malbec_out_layout(mb.OUT_FINAL, mb.FP64, 0, 10, 0, ctypes.byref(L)) == mb.EINVAL
    assert lib.malbec_out_layout(mb.OUT_STRIDED, mb.FP64, 10, 10, 0, ctypes.byref(L)) == mb.EINVAL
    assert lib.malbec_out_layout(7, mb.FP64, 10, 10, 1, ctypes.byref(L)) == mb.EINVAL
    assert lib.malbec_out_layout(mb.OUT_FINAL, 9, 10, 10, 1, ctypes.byref(L)) == mb.EINVAL
    assert lib.malbec_out_bytes(mb.OUT_STRIDED, mb.FP64, 1 << 30, 1 << 30, 1) == 0


def test_camera_layout(mb):
    cam = mb.make_camera(1000.0, 1.3, 25.0, 64, 48)
    L = mb.camera_layout(cam)
    n = 64 * 48
    assert L.fate % 256 == 0 and L.steps >= n and L.theta >= L.steps + 4 * n and L.phi >= L.theta + 8 * n
    assert L.total >= L.phi + 8 * n


def _term(**kw):
    from paper_1803_08320_gb300.malbec import Termination

    return Termination(**kw).c()


def test_trace_validation_rejects_before_any_cuda_call(mb):
    """Invalid physics is refused on the host (no device pointer is touched)."""
    lib = mb.lib()
    fake = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    good = _term(eps_hor=0.01, r_esc=1000.0, n_steps_cap=10, dl=0.01)
    cases = [
        (mb.Metric(1.0, 1.0, None), good),            # a = M
        (mb.Metric(1.0, 1.5, None), good),            # naked singularity (a > M, Sec. 2)
        (mb.Metric(0.0, 0.0, None), good),            # M <= 0
        (mb.Metric(1.0, -0.1, None), good),           # a < 0
        (mb.Metric(float("nan"), 0.0, None), good),
        (mb.Metric(1.0, 0.5, None), _term(dl=0.0)),   # no step
        (mb.Metric(1.0, 0.5, None), _term(dl=float("inf"))),
        (mb.Metric(1.0, 0.5, None), _term(dl=0.0, dl_r_scale=-0.05)),
        (mb.Metric(1.0, 0.5, None), _term(r_esc=1.5)),  # escape inside the capture radius
        (mb.Metric(1.0, 0.5, None), _term(eps_hor=-0.1)),
        (mb.Metric(1.0, 0.5, None), _term(form=3)),   # no such form
        (mb.Metric(1.0, 0.5, None), _term(method=2)),  # no such integrator
        (mb.Metric(1.0, 0.5, None), _term(method=1, rtol=1e-9, atol=0.0)),   # Dormand-Prince: atol > 0
        (mb.Metric(1.0, 0.5, None), _term(method=1, rtol=-1.0, atol=1e-9)),
        (mb.Metric(1.0, 0.5, None), _term(method=1, rtol=1e-9, atol=1e-9, dl=-1.0, dl_r_scale=0.5)),
    ]
    for m, t in cases:
        assert lib.malbec_trace(m, fake, 10, t, mb.OUT_FINAL, 0, mb.FP64, fake, None) == mb.EINVAL
    m = mb.Metric(1.0, 0.5, None)
    assert lib.malbec_trace(m, None, 10, good, mb.OUT_FINAL, 0, mb.FP64, fake, None) == mb.EINVAL
    assert lib.malbec_trace(m, fake, 0, good, mb.OUT_FINAL, 0, mb.FP64, fake, None) == mb.EINVAL
    assert lib.malbec_trace(m, fake, 10, good, mb.OUT_STRIDED, 0, mb.FP64, fake, None) == mb.EINVAL
    assert lib.malbec_trace(m, fake, 10, good, mb.OUT_FINAL, 0, mb.FP64, ctypes.c_void_p(257), None) == mb.EINVAL
    # Dormand-Prince in FP32_MIXED needs rtol >= MALBEC_DOPRI5_MIXED_RTOL_MIN (1e-6)
    for rtol in (1e-9, 0.99e-6):
        dp = _term(eps_hor=0.01, r_esc=1000.0, n_steps_cap=10, dl=0.01, method=1, rtol=rtol, atol=1e-9)
        assert lib.malbec_trace(m, fake, 10, dp, mb.OUT_FINAL, 0, mb.FP32_MIXED, fake, None) == mb.EINVAL
        cam = mb.make_camera(1000.0, 1.3, 25.0, 8, 8)
        assert lib.malbec_trace_camera(m, ctypes.byref(cam), dp, mb.FP32_MIXED, fake, None) == mb.EINVAL
        # and in the job tables (checked before anything is allocated or launched)
        b = mb.make_bundle(mb.BUNDLE_BOUND, 10, 1.0, 0.5, dp, seed=3)
        b.out = fake
        assert lib.malbec_trace_bundles(mb._bundle_array([b]), 1, mb.FP32_MIXED, None) == mb.EINVAL



def test_camera_validation(mb):
    lib = mb.lib()
    fake = ctypes.c_void_p(256)
    t = _term(eps_hor=0.01, r_esc=1100.0, n_steps_cap=100, dl=0.0, dl_r_scale=0.05)
    m = mb.Metric(1.0, 0.9, None)
    for cam in (mb.make_camera(1000.0, 0.0, 25.0, 8, 8),     # on the axis
                mb.make_camera(1000.0, 3.2, 25.0, 8, 8),
                mb.make_camera(1200.0, 1.3, 25.0, 8, 8),     # observer beyond r_esc
                mb.make_camera(1.0, 1.3, 25.0, 8, 8),        # inside the capture radius
                mb.make_camera(1000.0, 1.3, 0.0, 8, 8),
                mb.make_camera(1000.0, 1.3, 25.0, 0, 8)):
        assert lib.malbec_trace_camera(m, ctypes.byref(cam), t, mb.FP64, fake, None) == mb.EINVAL
    cam = mb.make_camera(1000.0, 1.3, 25.0, 8, 8)
    apr = mb.Metric(1.0, 0.9, ctypes.c_void_p(256))
    assert lib.malbec_trace_camera(apr, ctypes.byref(cam), t, mb.FP64, fake, None) == mb.EINVAL


def test_ic_validation(mb):
    lib = mb.lib()
    fake = ctypes.c_void_p(256)
    assert lib.malbec_ic_bound(1.0, 1.0, 0, 1, 0, 10, fake, fake, fake, None) == mb.EINVAL
    assert lib.malbec_ic_bound(1.0, 0.5, 0, 1, 0, 0, fake, fake, fake, None) == mb.EINVAL
    assert lib.malbec_ic_bound(1.0, 0.5, 0, 1, 1 << 60, 10, fake, fake, fake, None) == mb.EINVAL
    assert lib.malbec_ic_circular(mb.Metric(1.0, 0.0, None), None, 10, 1, fake, None) == mb.EINVAL
    assert lib.malbec_invariants(mb.Metric(1.0, 2.0, None), fake, 10, fake, None) == mb.EINVAL


def test_mixed_zone_setting(mb):
    z = mb.get_mixed_zone()
    assert (z.horizon_factor, z.photon_margin, z.pole_sin) == (2.0, 0.5, 0.2)
    z2 = mb.set_mixed_zone(pole_sin=0.25)
    assert z2.pole_sin == 0.25 and mb.get_mixed_zone().pole_sin == 0.25
    bad = mb.MixedZone(0.5, 0.5, 0.1)
    assert mb.lib().malbec_set_mixed_zone(ctypes.byref(bad)) == mb.EINVAL
    bad = mb.MixedZone(2.0, 0.5, 1.5)
    assert mb.lib().malbec_set_mixed_zone(ctypes.byref(bad)) == mb.EINVAL
    z3 = mb.set_mixed_zone(reset=True)
    assert (z3.horizon_factor, z3.photon_margin, z3.pole_sin) == (2.0, 0.5, 0.2)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1803_08320_gb300 import malbec

    monkeypatch.setattr(malbec, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(malbec, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        malbec.lib()


def test_cartesian_layout(mb):
    """MALBEC_OUT_STRIDED_CARTESIAN: the FINAL fields plus 4 components (t, x,
    y, z) per sample instead of 8."""
    n, cap, stride = 1000, 1000, 10
    L8 = mb.out_layout(mb.OUT_STRIDED, "fp64", n, cap, stride)
    L4 = mb.out_layout(mb.OUT_STRIDED_CARTESIAN, "fp64", n, cap, stride)
    assert L4.traj == L8.traj and L4.n_samples == L8.n_samples == cap // stride + 1
    assert L4.total - L4.traj == pytest.approx((L8.total - L8.traj) / 2, abs=256)
    L4f = mb.out_layout(mb.OUT_STRIDED_CARTESIAN, "fp32_mixed", n, cap, stride)
    assert L4f.total - L4f.traj >= n * L4f.n_samples * 16
    with pytest.raises(mb.MalbecError):
        mb.out_layout(mb.OUT_STRIDED_CARTESIAN, "fp64", n, cap, 0)


def test_launch_config_setting(mb):
    c = mb.get_launch_config()
    assert c.as_dict() == {"threads_per_block": 0, "blocks_per_sm": 0, "refill_min": 0, "zone_batch": 0,
                           "zone_wait": 0, "exchange": 0, "zone_wait_limit_us": 0}
    c2 = mb.set_launch_config(threads_per_block=64, blocks_per_sm=2, refill_min=4, zone_batch=8, zone_wait=32,
                              exchange=2, zone_wait_limit_us=1500)
    assert c2.as_dict() == {"threads_per_block": 64, "blocks_per_sm": 2, "refill_min": 4, "zone_batch": 8,
                            "zone_wait": 32, "exchange": 2, "zone_wait_limit_us": 1500}
    bad = mb.LaunchConfig(48, 0, 0, 0, 0)
    assert mb.lib().malbec_set_launch_config(ctypes.byref(bad)) == mb.EINVAL
    bad = mb.LaunchConfig(512, 0, 0, 0, 0)
    assert mb.lib().malbec_set_launch_config(ctypes.byref(bad)) == mb.EINVAL
    assert mb.set_launch_config(reset=True).as_dict()["threads_per_block"] == 0


def test_paper_rows_reader(mb, tmp_path):
    """The paper's initial-condition text layout (Sec. 5: t r theta phi p_t
    p_r p_theta p_phi per line): the three rows of the golden file parse to
    an (8, 3) array; a malformed line is an error."""
    import os

    rows = mb.read_paper_rows(os.path.join(os.path.dirname(__file__), "golden", "ic_rows.txt"))
    assert rows.shape == (8, 3) and rows.dtype == np.float64
    assert rows[1].tolist() == [6.0, 3.5, 4.0] and rows[4, 0] == 0.9428 and rows[7, 2] == 4.0
    bad = tmp_path / "bad.txt"
    bad.write_text("0 6 1.5708 0 0.9428 0 0\n")
    with pytest.raises(ValueError):
        mb.read_paper_rows(str(bad))


def test_ic_from_paper_validation(mb):
    lib = mb.lib()
    fake, other = ctypes.c_void_p(256), ctypes.c_void_p(512)
    good = mb.Metric(1.0, 0.0, None)
    assert lib.malbec_ic_from_paper(good, fake, 0, other, None) == mb.EINVAL
    assert lib.malbec_ic_from_paper(good, None, 3, other, None) == mb.EINVAL
    assert lib.malbec_ic_from_paper(good, fake, 3, fake, None) == mb.EINVAL   # rows and ics alias
    assert lib.malbec_ic_from_paper(mb.Metric(1.0, 1.0, None), fake, 3, other, None) == mb.EINVAL


def test_diagnostics_validate_before_any_cuda_call(mb):
    lib = mb.lib()
    v = ctypes.c_double()
    assert lib.malbec_measure_step_loop(7, ctypes.byref(v)) == mb.EINVAL
    assert lib.malbec_measure_step_loop(0, None) == mb.EINVAL
    assert lib.malbec_check_fp64_helpers(None) == mb.EINVAL
    assert lib.malbec_measure_fma_peak(5, ctypes.byref(v)) == mb.EINVAL


def test_binding_tensor_checks_reject_bad_buffers(mb):
    """The library sees raw pointers only, so the binding checks every buffer
    it hands over (device, dtype, contiguity, size) before any call; each bad
    case raises ValueError.  Checked here on CPU tensors with the device type
    the check expects set to "cpu"."""
    import torch

    chk = mb.check_device_tensor
    good = torch.zeros((8, 5), dtype=torch.float64)
    chk(good, "ics", torch.float64, shape=(8, 5), device_type="cpu")
    with pytest.raises(ValueError, match="float64"):
        chk(good.float(), "ics", torch.float64, device_type="cpu")
    with pytest.raises(ValueError, match="contiguous"):
        chk(torch.zeros((5, 8), dtype=torch.float64).t(), "ics", torch.float64, device_type="cpu")
    with pytest.raises(ValueError, match="shape"):
        chk(good, "ics", torch.float64, shape=(8, 6), device_type="cpu")
    with pytest.raises(ValueError, match="4 elements"):
        chk(torch.zeros(5, dtype=torch.float64), "a_per_ray", torch.float64, numel=4, device_type="cpu")
    with pytest.raises(ValueError, match="at least 1000"):
        chk(torch.zeros(999, dtype=torch.uint8), "out", torch.uint8, numel_min=1000, device_type="cpu")
    with pytest.raises(ValueError, match="cuda"):
        chk(good, "ics", torch.float64)
    with pytest.raises(ValueError, match="torch.Tensor"):
        chk(np.zeros((8, 5)), "ics", torch.float64, device_type="cpu")


def test_noalloc_binding_rejects_host_buffers_before_any_call(mb):
    """trace_noalloc never copies: host tensors are refused with ValueError
    (a raw host pointer handed to the kernel would fault)."""
    import torch

    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=10, dl=0.01)
    ics = torch.zeros((8, 4), dtype=torch.float64)
    out = torch.zeros(1 << 16, dtype=torch.uint8)
    with pytest.raises(ValueError, match="ics"):
        mb.trace_noalloc(1.0, 0.5, ics, t, out)

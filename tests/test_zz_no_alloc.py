"""malbec_trace_noalloc: the tracing entry point for callers that cannot
allocate device memory (graph capture that forbids allocation, real-time loops
that must stay out of the allocator, embedders that own all device memory).
It must give the same results as malbec_trace, call after call, while using
only the library's static work-queue block.  Collected last on purpose: a
failure here leaves every other test already run."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-9  # the tolerance of the FP64 parity tests


@pytest.fixture(scope="module")
def mb():
    import torch

    from paper_1803_08320_gb300 import build, malbec

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    malbec.lib()
    return malbec


def _close(a, b):
    """Within the parity tolerance, NaN matching NaN (a ray that ends
    NONFINITE has NaN components on both paths)."""
    a, b = a.cpu().numpy(), b.cpu().numpy()
    both_nan = np.isnan(a) & np.isnan(b)
    with np.errstate(invalid="ignore"):
        ok = np.abs(a - b) <= RTOL * np.maximum(np.abs(b), 1.0)
    return bool(np.all(ok | both_nan))


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_noalloc_matches_trace_on_two_calls_in_a_row(mb, precision):
    import torch

    from paper_1803_08320_gb300 import workloads as W

    wl = W.bound()
    ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, 3000)
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=2000, dl=0.02)
    ref = mb.trace(wl.M, 0.0, ics, t, precision=precision, a_per_ray=spins)
    L = mb.out_layout(mb.OUT_FINAL, precision, ics.shape[1], t.n_steps_cap, 0)
    # two calls in a row on different inputs: the second must not see the
    # first call's work-queue counter
    ics2, spins2, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, 1000, index0=50_000)
    ref2 = mb.trace(wl.M, 0.0, ics2, t, precision=precision, a_per_ray=spins2)
    out1 = torch.empty(L.total, dtype=torch.uint8, device="cuda")
    L2 = mb.out_layout(mb.OUT_FINAL, precision, ics2.shape[1], t.n_steps_cap, 0)
    out2 = torch.empty(L2.total, dtype=torch.uint8, device="cuda")
    got1 = mb.trace_noalloc(wl.M, 0.0, ics, t, out1, precision=precision, a_per_ray=spins)
    got2 = mb.trace_noalloc(wl.M, 0.0, ics2, t, out2, precision=precision, a_per_ray=spins2)
    torch.cuda.synchronize()
    for got, want in ((got1, ref), (got2, ref2)):
        assert _close(got["y"], want["y"])
        assert _close(got["inv1"], want["inv1"])
        assert torch.equal(got["fate"], want["fate"]) and torch.equal(got["steps"], want["steps"])


def test_noalloc_rejects_invalid_arguments(mb):
    fake = ctypes.c_void_p(256)
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=10, dl=0.01).c()
    lib = mb.lib()
    assert lib.malbec_trace_noalloc(mb.Metric(1.0, 1.0, None), fake, 10, t, mb.OUT_FINAL, 0, mb.FP64, fake,
                                    None) == mb.EINVAL
    assert lib.malbec_trace_noalloc(mb.Metric(1.0, 0.5, None), fake, 0, t, mb.OUT_FINAL, 0, mb.FP64, fake,
                                    None) == mb.EINVAL


def _default_pool_used_high():
    """USED_MEM_HIGH of the current device's default stream-ordered memory
    pool (driver API through ctypes), after resetting the watermark to the
    current use; returns (reset, read) callables."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used_high = 8  # CU_MEMPOOL_ATTR_USED_MEM_HIGH

    def reset():
        zero = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0

    def read():
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, used_high, ctypes.byref(v)) == 0
        return v.value

    return reset, read


def test_noalloc_takes_nothing_from_the_stream_ordered_pool(mb):
    """The property the entry point exists for: malbec_trace takes its
    work-queue block from the device's default stream-ordered pool (the
    watermark of the pool's used bytes rises), malbec_trace_noalloc takes
    nothing (the watermark stays where it was reset)."""
    import torch

    from paper_1803_08320_gb300 import workloads as W

    wl = W.bound()
    ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, 512)
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=200, dl=0.02)
    L = mb.out_layout(mb.OUT_FINAL, "fp64", 512, t.n_steps_cap, 0)
    out = torch.empty(L.total, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    reset, read = _default_pool_used_high()
    reset()
    base = read()
    mb.trace(wl.M, 0.0, ics, t, a_per_ray=spins)
    torch.cuda.synchronize()
    assert read() >= base + 256, "the control call should show its scratch block in the pool"
    torch.cuda.synchronize()
    reset()
    base = read()
    mb.trace_noalloc(wl.M, 0.0, ics, t, out, a_per_ray=spins)
    mb.trace_noalloc(wl.M, 0.0, ics, t, out, a_per_ray=spins)
    torch.cuda.synchronize()
    assert read() == base

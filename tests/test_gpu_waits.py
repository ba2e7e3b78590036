"""The bounded device-side wait of the trace kernels: the zone warp of an
FP32_MIXED block (block ray exchange on) waits, once it has no ray left, for
the other warps of its block, at most the launch configuration's
zone_wait_limit_us.  Here the limit is made to run out (1 us): the expiries
are counted and reported as MALBEC_ETIMEDOUT by malbec_wait_status, and every
ray's result is the same as with the default 2 s limit (the other warps take
their FP64-zone steps in place, with the same arithmetic)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    import torch

    from paper_1803_08320_gb300 import build, malbec

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    malbec.lib()
    yield malbec
    malbec.set_launch_config(reset=True)


def test_zone_warp_wait_runs_out_and_results_are_unchanged(mb):
    import torch

    from paper_1803_08320_gb300 import workloads as W

    wl = W.bound()
    # 128-thread blocks (the zone warp and three others), many rays per lane,
    # so that zone warps run out of rays while their block-mates still run
    ics, spins, _ = mb.ic_bound(wl.M, wl.a_max, wl.seed, 40_000)
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=1500, dl=0.02)
    mb.set_launch_config(threads_per_block=128, exchange=1)
    ref = mb.trace(wl.M, 0.0, ics, t, precision="fp32_mixed", a_per_ray=spins)
    torch.cuda.synchronize()
    mb.wait_status()  # forget earlier expiries
    mb.set_launch_config(threads_per_block=128, exchange=1, zone_wait_limit_us=1)
    got = mb.trace(wl.M, 0.0, ics, t, precision="fp32_mixed", a_per_ray=spins)
    timed_out, total = mb.wait_status()
    mb.set_launch_config(reset=True)
    assert timed_out and total > 0
    for k in ("y", "inv1", "lambda"):
        a, b = got[k], ref[k]
        assert torch.equal(torch.isnan(a), torch.isnan(b)), k
        assert torch.equal(torch.nan_to_num(a), torch.nan_to_num(b)), k
    assert torch.equal(got["fate"], ref["fate"]) and torch.equal(got["steps"], ref["steps"])
    # nothing ran out since: the status is back to OK
    assert mb.wait_status() == (False, total)

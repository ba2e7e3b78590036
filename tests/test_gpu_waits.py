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
    import numpy as np
    import torch

    # 40,000 rays, one in 64 a long circular orbit outside every FP64 zone
    # (r in [8, 12] M, equatorial: FP32 steps only), the others started
    # inside the capture radius (they end after one step).  With 128-thread
    # blocks (the zone warp and three others) and the exchange on, the zone
    # warp of a block whose long orbits sit in other warps runs out of rays
    # long before its block does.
    a, n = 0.5, 40_000
    rng = np.random.default_rng(17)
    long_idx = np.arange(0, n, 64)
    radii = rng.uniform(8.0, 12.0, len(long_idx))
    circ = mb.ic_circular(1.0, a, radii)
    ics = torch.zeros((8, n), dtype=torch.float64, device="cuda")
    ics[1] = 1.5                    # inside (1 + eps) r_+ = 1.885 M
    ics[2] = 1.0
    ics[4] = 1.0
    ics[:, torch.as_tensor(long_idx).cuda()] = circ
    t = mb.Termination(eps_hor=0.01, r_esc=1100.0, n_steps_cap=20_000, dl=0.02)
    mb.set_launch_config(threads_per_block=128, exchange=1)
    ref = mb.trace(1.0, a, ics, t, precision="fp32_mixed")
    torch.cuda.synchronize()
    mb.wait_status()  # forget earlier expiries
    mb.set_launch_config(threads_per_block=128, exchange=1, zone_wait_limit_us=1)
    got = mb.trace(1.0, a, ics, t, precision="fp32_mixed")
    timed_out, total = mb.wait_status()
    mb.set_launch_config(reset=True)
    assert timed_out and total > 0
    for k in ("y", "inv1", "lambda"):
        x, y = got[k], ref[k]
        assert torch.equal(torch.isnan(x), torch.isnan(y)), k
        assert torch.equal(torch.nan_to_num(x), torch.nan_to_num(y)), k
    assert torch.equal(got["fate"], ref["fate"]) and torch.equal(got["steps"], ref["steps"])
    assert int((got["steps"] == t.n_steps_cap).sum().item()) == len(long_idx)
    # nothing ran out since: the status is back to OK
    assert mb.wait_status() == (False, total)

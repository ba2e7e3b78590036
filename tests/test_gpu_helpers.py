"""FP64 helpers of the right-hand sides against CUDA's own results, and the
bare RK4 step-loop diagnostic.

The FP64 right-hand sides take one sincos per RK4 step and reach the later
stage angles by the angle-addition formulas with Taylor series for sin d and
cos d - 1, and replace the division by a refined hardware reciprocal.  Both
are checked here against CUDA's sincos and IEEE division on 2^22 seeded
inputs; the parity tests then check whole trajectories against the oracle."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mb():
    import torch

    from paper_1803_08320_gb300 import build, malbec

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    malbec.lib()
    return malbec


def test_trig_and_reciprocal_match_cuda(mb):
    e = mb.check_fp64_helpers()
    # |sin|, |cos| <= 1: 4 units in the last place of 1.0 at most
    assert e["sin_abs"] <= 4 * 2.0**-52, e
    assert e["cos_abs"] <= 4 * 2.0**-52, e
    # the refined reciprocal is within one unit in the last place of 1/x
    assert e["recip_ulp"] <= 1.0, e
    # the estimate it starts from is good to 2^-17 or better, so one cubic
    # step (error ~ estimate error cubed) reaches full precision
    assert e["recip_estimate_rel"] <= 2.0**-17, e
    # the steps' own sine and cosine (Cody-Waite reduction, Taylor series)
    # within 2 units of 2^-52 of CUDA's (each side within about one of the
    # exact value: measured 0.58 and 0.50 units against a long-double
    # reference on the host)
    assert e["step_sin_abs"] <= 2 * 2.0**-52, e
    assert e["step_cos_abs"] <= 2 * 2.0**-52, e


def test_step_loop_diagnostic(mb):
    rates = {f: mb.measure_step_loop(f) for f in (mb.FORM_GEODESIC, mb.FORM_HAMILTONIAN, mb.FORM_ADM)}
    assert all(v > 1e8 for v in rates.values()), rates
    # the canonical right-hand side is the cheapest of the three
    assert rates[mb.FORM_HAMILTONIAN] > rates[mb.FORM_GEODESIC], rates
    with pytest.raises(mb.MalbecError):
        mb.measure_step_loop(7)


def test_operand_forms_are_the_plain_operations_bit_for_bit(mb):
    """The FP64 kernels write x*y as fma(x, y, -0) and x + y as fma(x, 1, y)
    with the constants in per-thread registers (the form the GB300 FP64 unit
    takes at its full rate), double stage radii through the exponent field,
    and the FP32_MIXED step runs paired FP32 operations; each must give the
    IEEE result of the plain operation, signed zeros, subnormals, infinities
    and NaN included."""
    c = mb.check_operand_forms()
    assert all(v == 0 for v in c.values()), c

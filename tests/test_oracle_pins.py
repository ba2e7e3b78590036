"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every test here is CPU-only.  Each pins a part of the oracle to something other
than the oracle itself: values the paper prints (tests/golden/, each cited),
closed forms, exact invariants of the geodesic flow, independent quadratures,
textbook special cases, and brute-force criteria.  References are to Quiroga,
"MALBEC: a new CUDA-C ray-tracer in General Relativity", arXiv:1803.08320.
"""
import math

import numpy as np
import pytest
from conftest import load_golden

M1 = 1.0


def rng(seed=7):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------- metric
def test_metric_matches_adm_decomposition(orc):
    """Sec. 2: alpha, beta^phi, gamma_ij of Kerr reproduce eq. kerr through
    eq. ADM: g_tt = -alpha^2 + gamma_phph beta^2, g_tph = gamma_phph beta^phi,
    g_ij = gamma_ij.  The ADM expressions are separate formulas in the paper."""
    r_ = rng(1)
    for _ in range(50):
        a = r_.uniform(0, 0.999)
        r = r_.uniform(2.5, 50)
        th = r_.uniform(0.05, math.pi - 0.05)
        g = orc.metric(M1, a, r, th)
        al, be, ga = orc.adm(M1, a, r, th)
        assert g[0, 0] == pytest.approx(-al**2 + ga[2] * be**2, rel=1e-12, abs=1e-14)
        assert g[0, 3] == pytest.approx(ga[2] * be, rel=1e-12, abs=1e-15)
        assert g[1, 1] == pytest.approx(ga[0], rel=1e-14)
        assert g[2, 2] == pytest.approx(ga[1], rel=1e-14)
        assert g[3, 3] == pytest.approx(ga[2], rel=1e-14)


def test_metric_tphi_determinant_and_inverse(orc):
    """Closed-form identity of BL Kerr: g_tt g_phph - g_tph^2 = -Delta sin^2;
    and g g^{-1} = identity."""
    r_ = rng(2)
    for _ in range(50):
        a = r_.uniform(0, 0.999)
        r = r_.uniform(2.5, 50)
        th = r_.uniform(0.05, math.pi - 0.05)
        g = orc.metric(M1, a, r, th)
        gi = orc.inverse_metric(M1, a, r, th)
        Delta = r * r - 2 * r + a * a
        det = g[0, 0] * g[3, 3] - g[0, 3] ** 2
        assert det == pytest.approx(-Delta * math.sin(th) ** 2, rel=1e-11)
        np.testing.assert_allclose(g @ gi, np.eye(4), atol=1e-12)


def test_metric_derivatives_match_finite_differences(orc):
    """Analytic d_r g and d_theta g against 4th-order central differences."""
    r_ = rng(3)
    for _ in range(30):
        a = r_.uniform(0, 0.999)
        r = r_.uniform(2.5, 30)
        th = r_.uniform(0.1, math.pi - 0.1)
        dg = orc.metric_derivs(M1, a, r, th)
        for s, (dr, dth) in ((1, (1e-3 * r, 0)), (2, (0, 1e-3))):
            f = lambda k: orc.metric(M1, a, r + k * dr, th + k * dth)
            fd = (-f(2) + 8 * f(1) - 8 * f(-1) + f(-2)) / (12 * (dr + dth))
            np.testing.assert_allclose(dg[s], fd, rtol=1e-8, atol=1e-9 * np.abs(fd).max())
        assert np.all(dg[0] == 0) and np.all(dg[3] == 0)


def test_schwarzschild_christoffels_textbook(orc):
    """a = 0: the nine distinct non-zero Christoffel symbols of Schwarzschild
    (textbook values, e.g. Carroll ch. 5) and zeros elsewhere."""
    M = 1.3
    for r, th in ((7.0, 0.9), (3.1, 2.0), (40.0, 1.5)):
        G = orc.christoffel(M, 0.0, r, th)
        s, c = math.sin(th), math.cos(th)
        want = np.zeros((4, 4, 4))

        def put(m, a_, b, v):
            want[m, a_, b] = v
            want[m, b, a_] = v

        put(0, 0, 1, M / (r * (r - 2 * M)))
        put(1, 0, 0, M * (r - 2 * M) / r**3)
        put(1, 1, 1, -M / (r * (r - 2 * M)))
        put(1, 2, 2, -(r - 2 * M))
        put(1, 3, 3, -(r - 2 * M) * s * s)
        put(2, 1, 2, 1 / r)
        put(2, 3, 3, -s * c)
        put(3, 1, 3, 1 / r)
        put(3, 2, 3, c / s)
        np.testing.assert_allclose(G, want, rtol=1e-12, atol=1e-14)


def test_christoffel_symmetry_and_metric_compatibility(orc):
    """Gamma^m_{ab} = Gamma^m_{ba} and nabla g = 0:
    d_s g_{mn} = g_{ml} Gamma^l_{sn} + g_{nl} Gamma^l_{sm}."""
    r_ = rng(4)
    for _ in range(30):
        a = r_.uniform(0, 0.999)
        r = r_.uniform(2.5, 30)
        th = r_.uniform(0.1, math.pi - 0.1)
        G = orc.christoffel(M1, a, r, th)
        g = orc.metric(M1, a, r, th)
        dg = orc.metric_derivs(M1, a, r, th)
        np.testing.assert_allclose(G, np.transpose(G, (0, 2, 1)), atol=1e-15)
        lower = np.einsum("ml,lsn->smn", g, G)
        rhs = lower + np.transpose(lower, (0, 2, 1))
        np.testing.assert_allclose(rhs, dg, rtol=1e-10, atol=1e-12 * np.abs(dg).max())


# --------------------------------------------------------------------------- RHS
def _random_state(r_, a, r_lo=2.5, r_hi=40.0):
    r = r_.uniform(max(r_lo, 1 + math.sqrt(1 - a * a) + 0.3), r_hi)
    th = r_.uniform(0.2, math.pi - 0.2)
    u = r_.normal(size=4) * np.array([1.0, 0.3, 0.05, 0.05])
    u[0] = abs(u[0]) + 1.0
    return np.array([r_.uniform(0, 10), r, th, r_.uniform(0, 6), *u])


def test_rhs_matches_paper_schwarzschild_equations(orc):
    """Sec. 4: the Schwarzschild equations of motion in canonical form
    (t', r', th', ph', p_r', p_th'; p_t' = p_ph' = 0, paper p_t = +E),
    converted to du/dlambda, equal the oracle's Christoffel-form RHS at a = 0."""
    r_ = rng(5)
    M = 1.0
    for _ in range(40):
        y = _random_state(r_, 0.0)
        t, r, th, ph, ut, ur, uth, uph = y
        s, c = math.sin(th), math.cos(th)
        f0 = 1 - 2 * M / r
        E, pr, pth, pph = f0 * ut, ur / f0, r * r * uth, r * r * s * s * uph
        # the paper's right-hand sides
        tdot = E / f0
        rdot = f0 * pr
        thdot = pth / r**2
        phdot = pph / (r**2 * s**2)
        prdot = -M * E**2 / (-r + 2 * M) ** 2 - M * pr**2 / r**2 + pth**2 / r**3 + pph**2 / (r**3 * s**2)
        pthdot = pph**2 * c / (r**2 * s**3)
        # chain rule to the velocity form
        dut = -E * (2 * M / r**2) * rdot / f0**2
        dur = (2 * M / r**2) * rdot * pr + f0 * prdot
        duth = pthdot / r**2 - 2 * pth * rdot / r**3
        duph = -2 * pph * rdot / (r**3 * s**2) - 2 * pph * c * thdot / (r**2 * s**3)
        f = orc.rhs(M, 0.0, y)
        np.testing.assert_allclose(f[:4], [tdot, rdot, thdot, phdot], rtol=1e-13)
        np.testing.assert_allclose(f[4:], [dut, dur, duth, duph], rtol=1e-10,
                                   atol=1e-13 * np.abs(f[4:]).max())


def test_rhs_matches_paper_kerr_equatorial_equations(orc):
    """Sec. 3 eqs. dotr, dotphi, dotpr and the t' equation (equatorial Kerr,
    th = pi/2, th' = 0, paper p_t = +E).  t' and ph' depend on r only, so
    du^t/dl = (dt'/dr) r' and du^ph/dl = (dph'/dr) r' (4th-order differences);
    du^r/dl = d(Delta/r^2)/dr r' p_r + (Delta/r^2) p_r'; du^th/dl = 0."""
    r_ = rng(6)
    M = 1.0
    for _ in range(40):
        a = r_.uniform(0.0, 0.99)
        r0 = r_.uniform(3.0, 30.0)
        E = r_.uniform(0.8, 1.2)
        L = r_.uniform(-5, 5)
        pr = r_.uniform(-0.5, 0.5)
        w = lambda r: 2 * M * r - a * a - r * r

        def tdot(r):
            return (-(2 * M * a * a + a * a * r + r**3) * E + 2 * a * M * L) / (r * w(r))

        def phdot(r):
            return (-2 * M * a * E + (2 * M - r) * L) / (r * w(r))

        rdot = -w(r0) / r0**2 * pr
        prdot = (-(M * r0 - a * a) / r0**3 * pr**2
                 + M * (4 * M * a * a * r0 - a**4 - 2 * a * a * r0**2 - r0**4) / (r0**2 * w(r0) ** 2) * E**2
                 - 2 * M * a * (4 * M * r0 - a * a - 3 * r0**2) / (r0**2 * w(r0) ** 2) * E * L
                 + (4 * M * M * r0 - M * a * a - 4 * M * r0**2 + r0**3) / (r0**2 * w(r0) ** 2) * L**2)
        # state from the momenta through the oracle's own inverse metric
        y = orc.paper_to_state(M, a, [0, r0, math.pi / 2, 0, E, pr, 0, L])
        assert y[4] == pytest.approx(tdot(r0), rel=1e-12)
        assert y[7] == pytest.approx(phdot(r0), rel=1e-12, abs=1e-15)
        assert y[5] == pytest.approx(rdot, rel=1e-12, abs=1e-16)
        hh = 1e-3 * r0

        def d(fn):
            return (-fn(r0 + 2 * hh) + 8 * fn(r0 + hh) - 8 * fn(r0 - hh) + fn(r0 - 2 * hh)) / (12 * hh)

        Dr2 = lambda r: (r * r - 2 * M * r + a * a) / r**2
        want = [d(tdot) * rdot, d(Dr2) * rdot * pr + Dr2(r0) * prdot, 0.0, d(phdot) * rdot]
        f = orc.rhs(M, a, y)
        scale = np.abs(f[4:]).max()
        np.testing.assert_allclose(f[4:], want, rtol=1e-8, atol=1e-10 * scale)
        assert abs(f[6]) < 1e-14 * scale + 1e-300


def test_rhs_conserves_invariants_instantaneously(orc):
    """Exact first integrals of the geodesic flow: E = -p_t, L_z = p_ph, the
    norm g u u (eq. geo) and the Carter constant Q have zero derivative along
    the RHS.  A dropped term, wrong sign or index in any acceleration breaks
    at least one of these."""
    r_ = rng(8)
    for _ in range(60):
        a = r_.uniform(0.0, 0.999)
        y = _random_state(r_, a)
        f = orc.rhs(M1, a, y)
        eps = 1e-5
        dF = (orc.invariants(M1, a, y + eps * f) - orc.invariants(M1, a, y - eps * f)) / (2 * eps)
        # scale: derivative along a random direction of the same size
        v = r_.normal(size=8)
        v *= np.linalg.norm(f) / np.linalg.norm(v)
        dV = (orc.invariants(M1, a, y + eps * v) - orc.invariants(M1, a, y - eps * v)) / (2 * eps)
        scale = np.abs(dV) + np.abs(orc.invariants(M1, a, y)) * 1e-3 + 1e-12
        assert np.all(np.abs(dF) < 1e-6 * scale), (dF, scale)


def test_hamiltonian_cross_form(orc):
    """Sec. 2 eq. Ham: with p = g u, x' = g^{-1} p equals u, and p' equals
    d(g u)/dl computed from the Christoffel form (metric derivatives by finite
    differences, independent of the analytic ones)."""
    r_ = rng(9)
    for _ in range(30):
        a = r_.uniform(0.0, 0.999)
        y = _random_state(r_, a)
        p = orc.state_to_momenta(M1, a, y)
        fh = orc.rhs_hamiltonian(M1, a, np.concatenate([y[:4], p]))
        np.testing.assert_allclose(fh[:4], y[4:], rtol=1e-12, atol=1e-14)
        f = orc.rhs(M1, a, y)
        r, th = y[1], y[2]
        dr, dth = 1e-4 * r, 1e-4
        gr = (orc.metric(M1, a, r + dr, th) - orc.metric(M1, a, r - dr, th)) / (2 * dr)
        gth = (orc.metric(M1, a, r, th + dth) - orc.metric(M1, a, r, th - dth)) / (2 * dth)
        g = orc.metric(M1, a, r, th)
        pdot = (gr * y[5] + gth * y[6]) @ y[4:] + g @ f[4:]
        np.testing.assert_allclose(fh[4:], pdot, rtol=1e-6, atol=1e-7 * np.abs(pdot).max())


# --------------------------------------------------------------------------- RK4
def test_rk4_tableau_on_linear_ode(orc):
    """Classical RK4 on y' = lam y advances by exactly 1 + z + z^2/2 + z^3/6 + z^4/24."""
    for lam, h in ((-1.3, 0.1), (0.7, 0.25), (-20.0, 0.01)):
        z = lam * h
        got = orc.rk4_linear(lam, h, 1, 1.0)
        assert got == pytest.approx(1 + z + z * z / 2 + z**3 / 6 + z**4 / 24, rel=1e-15)
        got5 = orc.rk4_linear(lam, h, 5, 2.0)
        assert got5 == pytest.approx(2.0 * (1 + z + z * z / 2 + z**3 / 6 + z**4 / 24) ** 5, rel=1e-14)


def test_self_convergence_coefficient_is_16(orc):
    """Sec. 6.3 eq. Qt: Q = |y_h - y_{h/2}| / |y_{h/2} - y_{h/4}| ~ 2^4 for RK4,
    Euclidean norm over the 8 components, 10 random timelike Kerr a = 0.5
    geodesics (the generic bound-orbit sampler with the spin fixed at 0.5)."""
    h = 0.4
    n_out = 40
    Qs = []
    for idx in range(10):
        y0 = orc.bound_sample(M1, 0.5, 99, idx, spin_fixed=True)["y"]
        trajs = []
        for k in (1, 2, 4):
            term = orc.make_term(n_steps_cap=n_out * 10 * k, dl=h / k, r_esc=1e9)
            trajs.append(orc.trace_one(M1, 0.5, y0, term, stride=10 * k)["traj"])
        d1 = np.linalg.norm(trajs[0] - trajs[1], axis=1)[1:]
        d2 = np.linalg.norm(trajs[1] - trajs[2], axis=1)[1:]
        Qs.append(d1 / d2)
    Qs = np.array(Qs)
    assert 14.5 < np.median(Qs) < 17.5, np.median(Qs)
    assert np.percentile(Qs, 10) > 12.0


def test_radial_infall_cycloid_and_h4_error(orc):
    """Schwarzschild radial infall from rest at r0 (textbook closed form):
    r = r0 (1 + cos eta)/2, tau = sqrt(r0^3 / 8M) (eta + sin eta).  The RK4
    error against it shrinks by 2^4 when h is halved (fourth order).  (A
    circular orbit cannot show this: it is an equilibrium of the r, theta, u
    equations, which RK4 reproduces to rounding.)"""
    from scipy.optimize import brentq

    M, r0, tau_end = 1.0, 20.0, 80.0
    y0 = np.array([0, r0, math.pi / 2, 0, 1 / math.sqrt(1 - 2 * M / r0), 0, 0, 0])
    assert orc.invariants(M, 0.0, y0)[3] == pytest.approx(-1.0, abs=1e-15)
    k = math.sqrt(r0**3 / (8 * M))
    eta = brentq(lambda e: k * (e + math.sin(e)) - tau_end, 0.0, math.pi)
    r_exact = r0 * (1 + math.cos(eta)) / 2
    errs = []
    for h in (0.8, 0.4, 0.2):
        out = orc.trace_one(M, 0.0, y0, orc.make_term(n_steps_cap=int(round(tau_end / h)), dl=h))
        errs.append(abs(out["y"][1] - r_exact))
    assert errs[2] < 1e-6
    assert 13 < errs[0] / errs[1] < 19 and 13 < errs[1] / errs[2] < 19, errs


# --------------------------------------------------------------------------- circular orbits
def test_ic_rows_from_gralorbits(orc):
    """Sec. 5 ic.txt rows (4 dp) equal eq. gralorbits at k = 6, 3.5, 4, and
    each row satisfies the timelike constraint 2L = -1 (eq. geo) to the
    4-digit rounding."""
    rows = np.array(load_golden("ic_rows.txt"), dtype=float)
    for row, k in zip(rows, (6.0, 3.5, 4.0)):
        pt, pph = orc.schw_gralorbits(k, 1.0)
        assert row[1] == k
        assert abs(row[4] - pt) <= 5e-5 and abs(row[7] - pph) <= 5e-5
        y = orc.paper_to_state(1.0, 0.0, row)
        assert abs(orc.invariants(1.0, 0.0, y)[3] + 1) < 2e-3
        # full-precision values satisfy it to rounding
        y = orc.paper_to_state(1.0, 0.0, [0, k, math.pi / 2, 0, pt, 0, 0, pph])
        assert orc.invariants(1.0, 0.0, y)[3] == pytest.approx(-1.0, abs=1e-14)


def test_schwarzschild_isco_and_photon_sphere(orc):
    """Sec. 4: eqs. COrbit/COrbit2 give E = sqrt(8/9), L = sqrt(12) M at the
    ISCO r = 6M (eq. isco); |dE/dr| = M|6M - r|/(2 r^{3/2}(r - 3M)^{3/2}) with
    its only root at 6M (the paper prints the opposite sign: E grows towards 1
    for r > 6M; the sign here follows the mathematics); E diverges as r -> 3M (no circular timelike
    orbit inside the photon sphere)."""
    E, L = orc.schw_circular(1.0, 6.0)
    assert E == pytest.approx(math.sqrt(8 / 9), rel=1e-15)
    assert L == pytest.approx(math.sqrt(12), rel=1e-15)
    for M in (1.0, 2.5):
        for r in (6.5 * M, 9 * M, 25 * M):
            h = 1e-5 * r
            dE = (orc.schw_circular(M, r + h)[0] - orc.schw_circular(M, r - h)[0]) / (2 * h)
            assert dE == pytest.approx(-M * (6 * M - r) / (2 * r**1.5 * (r - 3 * M) ** 1.5), rel=1e-7)
            assert dE > 0
        assert orc.schw_circular(M, 3 * M * (1 + 1e-10))[0] > 1e4
    assert orc.photon_orbit(1.0, 0.0, 1) == pytest.approx(3.0, rel=1e-15)
    assert orc.photon_orbit(1.0, 0.0, 0) == pytest.approx(3.0, rel=1e-15)


@pytest.mark.parametrize("fname,prograde", [("isco_corotating.txt", 1), ("isco_counterrotating.txt", 0)])
def test_kerr_isco_tables(orc, fname, prograde):
    """Sec. 6.2 Tables ISCO-Co / ISCO-Count: Bardeen-Press-Teukolsky ISCO
    radius and the energy/angular momentum there reproduce the printed digits.
    The a = 1 co-rotating row is the limit r -> M+."""
    for a, r_t, pt_t, pph_t in np.array(load_golden(fname), dtype=float):
        r = orc.isco_bardeen(1.0, a, prograde)
        if a == 1.0 and prograde:
            assert r == pytest.approx(1.0, abs=1e-12)
            E, L = orc.kerr_circular_bardeen(1.0, a, 1.0 + 1e-5, prograde)
            assert E == pytest.approx(pt_t, abs=1e-3) and L == pytest.approx(pph_t, abs=1e-3)
            continue
        # the printed radii carry 12 decimals but agree with the closed form to
        # ~5e-11 (worst row a = 0.8); E and L are stationary at the ISCO
        assert r == pytest.approx(r_t, abs=1e-10)
        E, L = orc.kerr_circular_bardeen(1.0, a, r, prograde)
        assert E == pytest.approx(pt_t, abs=2e-12)
        assert L == pytest.approx(pph_t, abs=2e-11)
        # eq. ISCO: the ISCO is where dE/dr = 0
        assert orc.dEdr_root(1.0, a, prograde, r - 0.5 * (r - 1), r + 1.0) == pytest.approx(r, rel=1e-7)


def test_kerr_a05_quoted_iscos(orc):
    """Sec. 6.2: the 13-digit ISCO initial conditions quoted for a = 0.5."""
    for sg, r_t, pt_t, pph_t in np.array(load_golden("kerr_a05_isco.txt"), dtype=float):
        pro = int(sg > 0)
        r = orc.isco_bardeen(1.0, 0.5, pro)
        E, L = orc.kerr_circular_bardeen(1.0, 0.5, r, pro)
        assert r == pytest.approx(r_t, abs=2e-12)
        assert E == pytest.approx(pt_t, abs=2e-13)
        assert L == pytest.approx(pph_t, abs=2e-12)


def test_extreme_kerr_limits(orc):
    """Sec. 3 eqs. exKerr+/-: a -> M gives r+ = M, L+ = 2M/sqrt3 and
    r- = 9M, L- = -22M/(3 sqrt3), E- = 5/(3 sqrt3).  eq. exKerr+ prints
    E+ = 1/3 but Table ISCO-Co lists 0.5773502691896 = 1/sqrt3 (Bardeen); the
    oracle follows the table."""
    a = 1.0
    assert orc.isco_bardeen(1.0, a, 0) == pytest.approx(9.0, abs=1e-12)
    E, L = orc.kerr_circular_bardeen(1.0, a, 9.0, 0)
    assert E == pytest.approx(5 / (3 * math.sqrt(3)), rel=1e-14)
    assert L == pytest.approx(-22 / (3 * math.sqrt(3)), rel=1e-14)
    E, L = orc.kerr_circular_bardeen(1.0, a, 1.0 + 1e-5, 1)
    assert E == pytest.approx(1 / math.sqrt(3), abs=1e-3)
    assert L == pytest.approx(2 / math.sqrt(3), abs=1e-3)
    table_E = float(load_golden("isco_corotating.txt")[-1][2])
    assert table_E == pytest.approx(1 / math.sqrt(3), abs=1e-12)
    assert abs(table_E - 1 / 3) > 0.2


def test_paper_energy_momentum_branch_labels(orc):
    """Sec. 3 eqs. energia/momento as printed: the '+' branch (the paper calls
    it co-rotating) reproduces the counter-rotating Bardeen E with the sign of
    L flipped, and the same formula with a -> -a reproduces the co-rotating
    values: the printed labels are swapped."""
    for a in (0.1, 0.3, 0.5, 0.8, 0.95):
        for r in (orc.isco_bardeen(1, a, 0), 12.0, 20.0):
            Eb, Lb = orc.kerr_circular_bardeen(1.0, a, r, 0)
            Ep, Lp = orc.kerr_circular_paper(1.0, a, r, +1)
            assert Ep == pytest.approx(Eb, rel=1e-12) and Lp == pytest.approx(-Lb, rel=1e-12)
        for r in (orc.isco_bardeen(1, a, 1), 12.0, 20.0):
            Eb, Lb = orc.kerr_circular_bardeen(1.0, a, r, 1)
            Ep, Lp = orc.kerr_circular_paper(1.0, -a, r, +1)
            assert Ep == pytest.approx(Eb, rel=1e-12) and Lp == pytest.approx(Lb, rel=1e-12)


def test_paper_isco_closed_form_is_garbled(orc):
    """Sec. 3 eq. iscokerr evaluated literally takes the root of a negative
    number at a = 0.1, 0.5, 0.9; the oracle uses Bardeen's closed form instead."""
    for a in (0.1, 0.5, 0.9):
        assert math.isnan(orc.isco_paper_literal(1.0, a, 1))
        assert math.isnan(orc.isco_paper_literal(1.0, a, -1))


def test_circular_orbits_stay_closed_schwarzschild(orc):
    """Sec. 4 / Sec. 6.1: stable circular orbits keep r = r0 and phi = omega tau
    with omega = p_ph / r^2 (period T = 2 pi r^2 / p_ph), t = u^t tau, over
    10^4 steps of dtau = 0.01."""
    for r0 in (6.5, 10.0, 20.0):
        E, L = orc.schw_circular(1.0, r0)
        y0 = orc.paper_to_state(1.0, 0.0, [0, r0, math.pi / 2, 0, E, 0, 0, L])
        out = orc.trace_one(1.0, 0.0, y0, orc.make_term(n_steps_cap=10_000, dl=0.01), stride=1000)
        tr = out["traj"]
        tau = np.arange(tr.shape[0]) * 10.0
        assert np.abs(tr[:, 1] - r0).max() < 1e-9 * r0
        np.testing.assert_allclose(tr[:, 3], L / r0**2 * tau, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(tr[:, 0], y0[4] * tau, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(tr[:, 2], math.pi / 2, atol=1e-15)
        assert out["fate"] == orc.FATE_CAPPED and out["steps"] == 10_000


def test_circular_orbits_stay_closed_kerr(orc):
    """Sec. 3 eq. omega: a circular equatorial Kerr orbit (a = 0.5, co- and
    counter-rotating, outside the ISCO) keeps r and advances
    phi = omega tau with omega from the paper's formula (paper p_t = E)."""
    a = 0.5
    for r0, pro in ((5.0, 1), (8.0, 1), (9.0, 0), (12.0, 0)):
        E, L = orc.kerr_circular_bardeen(1.0, a, r0, pro)
        om = orc.kerr_omega(1.0, a, r0, E, L)
        y0 = orc.circular_state(1.0, a, r0, pro)
        out = orc.trace_one(1.0, a, y0, orc.make_term(n_steps_cap=5000, dl=0.02), stride=500)
        tr = out["traj"]
        tau = np.arange(tr.shape[0]) * 10.0
        assert np.abs(tr[:, 1] - r0).max() < 1e-8 * r0
        np.testing.assert_allclose(tr[:, 3], om * tau, rtol=1e-9, atol=1e-12)


def test_output_table_two_steps(orc):
    """Sec. 5 output.txt rows: RK4 with h = 0.1 from the r = 6 and r = 3.5
    circular Schwarzschild orbits, mapped to Cartesian by eq. coord, gives
    (tau, t, x, y, z) to the four printed decimals."""
    rows = np.array(load_golden("output_rows.txt"), dtype=float)
    ys = {}
    for pid, k in ((1, 6.0), (2, 3.5)):
        pt, pph = orc.schw_gralorbits(k, 1.0)
        ys[pid] = orc.paper_to_state(1.0, 0.0, [0, k, math.pi / 2, 0, pt, 0, 0, pph])
    states = {pid: [ys[pid]] for pid in ys}
    for pid in ys:
        y = ys[pid]
        for _ in range(2):
            y = orc.rk4_step(1.0, 0.0, 0.1, y)
            states[pid].append(y)
    for pid, tau, t, x, yy, z in rows:
        st = states[int(pid)][int(round(tau / 0.1))]
        xyz = orc.bl_to_cartesian(0.0, st[1], st[2], st[3])
        assert abs(st[0] - t) <= 5.1e-5
        np.testing.assert_allclose(xyz, [x, yy, z], atol=5.1e-5)


def _circ_traj(orc, a, r0, pro, h, tau, delta=1e-6):
    """Circular orbit with u^phi perturbed by a relative delta (the paper's
    initial conditions carry the rounding of E and L; an exactly circular
    state is an equilibrium of the r, theta, u equations and of RK4)."""
    y0 = orc.circular_state(1.0, a, r0, pro)
    y0[7] *= 1.0 + delta
    n = int(round(tau / h))
    stride = int(round(1.0 / h))
    out = orc.trace_one(1.0, a, y0, orc.make_term(n_steps_cap=n, dl=h, r_esc=1e3), stride=stride)
    return out["traj"]


def _dev(tr, r0):
    r = tr[np.isfinite(tr[:, 1]), 1]
    return np.abs(r - r0).max()


def test_stability_regions(orc):
    """Sec. 4 / Sec. 6.1-6.2 (Figs. 1-6): perturbed circular orbits between the
    photon orbit and the ISCO leave their radius, orbits outside the ISCO keep
    it; the trajectory of an unstable orbit depends on h (Fig. 3) far more than
    that of a stable orbit (Fig. 4)."""
    # Schwarzschild: 3M < r < 6M unstable, r > 6M stable
    tu1 = _circ_traj(orc, 0.0, 4.0, 1, 0.1, 2000.0)
    ts1 = _circ_traj(orc, 0.0, 8.0, 1, 0.1, 2000.0)
    assert _dev(tu1, 4.0) > 0.1 and _dev(ts1, 8.0) < 1e-3
    tu2 = _circ_traj(orc, 0.0, 4.0, 1, 0.05, 2000.0)
    ts2 = _circ_traj(orc, 0.0, 8.0, 1, 0.05, 2000.0)
    both = np.isfinite(tu1[:, 1]) & np.isfinite(tu2[:, 1])
    d_unstable = np.abs(tu1[both, 1] - tu2[both, 1]).max()
    d_stable = np.abs(ts1[:, 1] - ts2[:, 1]).max()
    assert d_unstable > 1e3 * d_stable, (d_unstable, d_stable)
    # Kerr a = 0.5: inside / outside the co- (4.233) and counter-rotating (7.555) ISCO
    assert _dev(_circ_traj(orc, 0.5, 3.6, 1, 0.1, 2000.0), 3.6) > 0.1
    assert _dev(_circ_traj(orc, 0.5, 5.0, 1, 0.1, 2000.0), 5.0) < 1e-3
    assert _dev(_circ_traj(orc, 0.5, 6.5, 0, 0.1, 2000.0), 6.5) > 0.1
    assert _dev(_circ_traj(orc, 0.5, 9.0, 0, 0.1, 2000.0), 9.0) < 1e-3


# --------------------------------------------------------------------------- null rays
def _equatorial_null(orc, a, r0, b, inward=True):
    """Equatorial null ray with E = 1, L = b at r0, via p_r from H = 0."""
    gi = orc.inverse_metric(1.0, a, r0, math.pi / 2)
    p = np.array([-1.0, 0.0, 0.0, b])
    rest = gi[0, 0] * p[0] ** 2 + 2 * gi[0, 3] * p[0] * p[3] + gi[3, 3] * p[3] ** 2
    pr = math.sqrt(max(-rest / gi[1, 1], 0.0)) * (-1 if inward else 1)
    p[1] = pr
    return np.concatenate([[0, r0, math.pi / 2, 0], gi @ p])


def test_schwarzschild_critical_impact_parameter(orc):
    """Photon sphere r = 3M and critical impact parameter 3 sqrt(3) M: rays
    from r = 1000 M with b < 3 sqrt3 are captured, with b > 3 sqrt3 escape;
    the circular photon orbit r = 3M, b = 3 sqrt3 M stays at r = 3M."""
    bc = 3 * math.sqrt(3)
    term = orc.make_term(eps_hor=0.01, r_esc=1100.0, n_steps_cap=20_000, dl=0.0, dl_r_scale=0.01)
    for b, fate in ((bc - 0.2, orc.FATE_CAPTURED), (bc - 0.02, orc.FATE_CAPTURED),
                    (bc + 0.02, orc.FATE_ESCAPED), (bc + 0.2, orc.FATE_ESCAPED)):
        assert orc.trace_one(1.0, 0.0, _equatorial_null(orc, 0.0, 1000.0, b), term)["fate"] == fate
    y0 = np.array([0, 3.0, math.pi / 2, 0, 0, 0, 0, 0.0])
    y0[4:] = orc.inverse_metric(1.0, 0.0, 3.0, math.pi / 2) @ np.array([-1.0, 0, 0, bc])
    assert orc.invariants(1.0, 0.0, y0)[3] == pytest.approx(0.0, abs=1e-15)
    out = orc.trace_one(1.0, 0.0, y0, orc.make_term(n_steps_cap=200, dl=0.01), stride=1)
    assert np.abs(out["traj"][:, 1] - 3.0).max() < 1e-9


def test_kerr_equatorial_photon_orbits(orc):
    """Bardeen photon-orbit radii r_ph = 2M(1 + cos(2/3 arccos(-+a/M))) and
    the critical-curve constant xi(r) = L/E agree: the photon with L = xi(r_ph)
    at r_ph has H = 0 with p_r = 0 (a circular null orbit) and stays there."""
    for a in (0.3, 0.9, 0.998):
        for pro in (1, 0):
            r = orc.photon_orbit(1.0, a, pro)
            xi = (r * r * (3 - r) - a * a * (r + 1)) / (a * (r - 1))
            y0 = np.zeros(8)
            y0[1], y0[2] = r, math.pi / 2
            y0[4:] = orc.inverse_metric(1.0, a, r, math.pi / 2) @ np.array([-1.0, 0, 0, xi])
            assert orc.invariants(1.0, a, y0)[3] == pytest.approx(0.0, abs=1e-12)
            out = orc.trace_one(1.0, a, y0, orc.make_term(n_steps_cap=100, dl=0.005), stride=1)
            assert np.abs(out["traj"][:, 1] - r).max() < 1e-8


def _deflection_quadrature(b, r_start, r_end):
    """Exact change of phi of a Schwarzschild null ray (M = 1) with impact
    parameter b from r_start inward to periapsis and out to r_end:
    dphi = int du / sqrt(1/b^2 - u^2 + 2u^3), u = 1/r, with u = u_max - s^2."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    f = lambda u: 1 / b**2 - u * u + 2 * u**3
    umax = brentq(f, 0.0, 1 / 3, xtol=1e-300, rtol=4 * np.finfo(float).eps)  # periapsis 1/r_min
    # f(u) = (u - umax) P(u) with P(u) = 2u^2 + (2 umax - 1) u + 2 umax^2 - umax;
    # u = umax - s^2 turns the integrand into 2 / sqrt(-P(umax - s^2)), regular at s = 0
    P = lambda u: 2 * u * u + (2 * umax - 1) * u + 2 * umax * umax - umax

    def piece(r):
        smax = math.sqrt(umax - 1 / r)
        g = lambda s: 2.0 / math.sqrt(-P(umax - s * s))
        return quad(g, 0.0, smax, epsabs=1e-15, epsrel=1e-13, limit=200)[0]

    return piece(r_start) + piece(r_end)


def test_null_deflection_matches_quadrature_and_weak_field(orc):
    """Schwarzschild null deflection: the oracle's phi change between r = R
    (in) and the escape radius (out) equals the exact quadrature; for large b
    the total bending approaches 4M/b + 15 pi M^2 / (4 b^2)."""
    R = 2.0e4
    for b in (30.0, 200.0):
        y0 = _equatorial_null(orc, 0.0, R, b)
        term = orc.make_term(eps_hor=0.01, r_esc=R, n_steps_cap=200_000, dl=0.0, dl_r_scale=2e-3)
        out = orc.trace_one(1.0, 0.0, y0, term)
        assert out["fate"] == orc.FATE_ESCAPED
        exact = _deflection_quadrature(b, R, out["y"][1])
        assert out["y"][3] == pytest.approx(exact, rel=2e-9)
        # weak field: the quadrature from infinity to infinity
        total = _deflection_quadrature(b, 1e12, 1e12) - math.pi
        approx2 = 4 / b + 15 * math.pi / (4 * b * b)
        assert abs(total - approx2) < 50 / b**3


def test_camera_initial_conditions(orc):
    """Backward camera (not in the paper): H = 0 at the observer, and the reversed
    ray carries E = -1, L_z = alpha sin th_o, Q = beta^2 + cos^2 th_o (alpha^2 - a^2)
    (Carter's constant is even in p), moving inward."""
    a, r_o, th_o, fov, nx, ny = 0.9, 1000.0, math.radians(80), 25.0, 64, 48
    for pix in (0, 17, nx * ny // 2 + 5, nx * ny - 1, 1234):
        y = orc.camera_ic(1.0, a, r_o, th_o, fov, nx, ny, pix)
        i, j = pix % nx, pix // nx
        al = -fov + 2 * fov * (i + 0.5) / nx
        be = -fov + 2 * fov * (j + 0.5) / ny
        E, Lz, Q, norm = orc.invariants(1.0, a, y)
        assert E == pytest.approx(-1.0, rel=1e-12)
        assert Lz == pytest.approx(al * math.sin(th_o), rel=1e-10, abs=1e-12)
        assert Q == pytest.approx(be * be + math.cos(th_o) ** 2 * (al * al - a * a), rel=1e-8, abs=1e-9)
        assert abs(norm) < 1e-13
        assert y[5] < 0 and y[1] == r_o and y[2] == th_o and y[0] == 0 and y[3] == 0


def _captured_by_potential(a, Lz, Q, r_lo, r_hi=1000.0):
    """Brute force: an ingoing photon (E = 1) is captured iff the radial
    potential R(r) stays positive between the horizon and the observer."""
    r = np.geomspace(r_lo, r_hi, 200_000)
    Delta = r * r - 2 * r + a * a
    R = ((r * r + a * a) - a * Lz) ** 2 - Delta * (Q + (Lz - a) ** 2)
    return bool(np.all(R > 0))


def test_camera_fates_match_radial_potential(orc):
    """Pixel fate of the oracle's backward integration equals the brute-force
    capture criterion on the radial potential, away from the critical curve
    (distance > 0.15M), for a = 0.9, th_o = 80 deg on a coarse grid."""
    a, r_o, th_o, fov, nx, ny = 0.9, 1000.0, math.radians(80), 12.0, 24, 24
    term = orc.make_term(eps_hor=0.01, r_esc=1100.0, n_steps_cap=20_000, dl=0.0, dl_r_scale=0.05)
    rp = orc.r_plus(1.0, a)
    checked = 0
    for pix in range(nx * ny):
        i, j = pix % nx, pix // nx
        al = -fov + 2 * fov * (i + 0.5) / nx
        be = -fov + 2 * fov * (j + 0.5) / ny
        if orc.critical_curve_distance(1.0, a, th_o, al, be) < 0.15:
            continue
        y = orc.camera_ic(1.0, a, r_o, th_o, fov, nx, ny, pix)
        out = orc.trace_one(1.0, a, y, term)
        Lz = -al * math.sin(th_o)
        Q = be * be + math.cos(th_o) ** 2 * (al * al - a * a)
        want = orc.FATE_CAPTURED if _captured_by_potential(a, Lz, Q, 1.01 * rp) else orc.FATE_ESCAPED
        assert out["fate"] & orc.FATE_MASK == want, (pix, al, be, out)
        checked += 1
    assert checked > 0.8 * nx * ny


def _min_radial_potential(a, Lz, Q, r_lo, r_hi=60.0):
    """Smallest value of the photon radial potential (E = 1)
    R(r) = ((r^2 + a^2) - a L_z)^2 - Delta (Q + (L_z - a)^2) on [r_lo, r_hi]:
    a dense grid, then a bounded scalar minimisation around the grid minimum.
    Beyond 60 M, R ~ r^4 stays positive for the impact parameters used here."""
    from scipy.optimize import minimize_scalar

    def R(r):
        Delta = r * r - 2 * r + a * a
        return ((r * r + a * a) - a * Lz) ** 2 - Delta * (Q + (Lz - a) ** 2)

    r = np.linspace(r_lo, r_hi, 6000)
    k = int(np.argmin(R(r)))
    lo, hi = r[max(k - 1, 0)], r[min(k + 1, len(r) - 1)]
    res = minimize_scalar(R, bounds=(lo, hi), method="bounded", options={"xatol": 1e-13})
    return min(float(res.fun), float(R(r[k])))


def _shadow_edge(a, th_o, centre, phi, t_max=15.0):
    """Point of the capture boundary on the ray centre + t (cos phi, sin phi):
    the zero of t -> min_r R(r; L_z, Q), positive while the photon is captured
    (R stays positive down to the horizon) and negative once it has a turning
    point; L_z = -alpha sin th_o, Q = beta^2 + cos^2 th_o (alpha^2 - a^2)."""
    from scipy.optimize import brentq

    r_lo = 1.0 + math.sqrt(1.0 - a * a)
    so, co = math.sin(th_o), math.cos(th_o)

    def g(t):
        al = centre[0] + t * math.cos(phi)
        be = centre[1] + t * math.sin(phi)
        return _min_radial_potential(a, -al * so, be * be + co * co * (al * al - a * a), r_lo)

    assert g(0.0) > 0 and g(t_max) < 0
    t = brentq(g, 0.0, t_max, xtol=1e-13, rtol=1e-15, maxiter=200)
    return centre[0] + t * math.cos(phi), centre[1] + t * math.sin(phi)


@pytest.mark.parametrize("a,incl_deg", [(0.9, 80.0), (0.5, 30.0), (0.998, 60.0)])
def test_critical_curve_distance_on_the_capture_boundary(orc, a, incl_deg):
    """The critical curve (Bardeen's xi(r), eta(r) of the spherical photon
    orbits) is the edge of the set of impact parameters whose photons the
    black hole captures.  That edge is found here without the curve's
    formulas: along 16 rays from a captured centre, the zero of min_r R(r) of
    the radial potential; the oracle's distance from every such point to its
    curve must vanish (a 1% error in xi or eta moves the curve by about
    0.03-0.07 M and fails this)."""
    th_o = math.radians(incl_deg)
    centre = (2.0 * a * math.sin(th_o), 0.0)  # inside the shadow (shifted towards retrograde alpha > 0)
    worst = 0.0
    for k in range(16):
        phi = (k + 0.5) * 2 * math.pi / 16
        al, be = _shadow_edge(a, th_o, centre, phi)
        d = orc.critical_curve_distance(1.0, a, th_o, al, be)
        worst = max(worst, d)
    assert worst < 1e-5, worst


def test_critical_curve_distance_at_the_equatorial_photon_orbits(orc):
    """Edge-on observer (th_o = 90 deg): the curve crosses beta = 0 at
    alpha = -b, b = L/E of the prograde and retrograde circular equatorial
    photon orbits.  b follows from R(r) = 0 on Q = 0 at the photon-orbit radius
    (Bardeen's r_ph, pinned against the paper's photon orbits above):
    r^2 + a^2 - a b = s sqrt(Delta) (b - a), so
    b = (r^2 + a^2 + s a sqrt(Delta)) / (a + s sqrt(Delta)); R'(r) = 0 there
    is checked too.  Schwarzschild's circle of radius 3 sqrt(3) M is the a = 0
    case."""
    th_o = math.pi / 2
    assert orc.critical_curve_distance(1.0, 0.0, th_o, 3 * math.sqrt(3.0), 0.0) < 1e-12
    for a in (0.3, 0.7, 0.9, 0.998):
        for prograde, s in ((1, 1.0), (0, -1.0)):
            r = orc.photon_orbit(1.0, a, prograde)
            Delta = r * r - 2 * r + a * a
            sD = math.sqrt(Delta)
            b = (r * r + a * a + s * a * sD) / (a + s * sD)
            dR = 4 * r * (r * r + a * a - a * b) - (2 * r - 2) * (b - a) ** 2
            assert abs(dR) < 1e-9 * (1 + abs(b)) ** 2 * r
            assert (b > 0) == bool(prograde)
            assert orc.critical_curve_distance(1.0, a, th_o, -b, 0.0) < 1e-5
            # a point 1% further out along alpha is about 0.01 |b| away
            assert orc.critical_curve_distance(1.0, a, th_o, -1.01 * b, 0.0) > 0.004 * abs(b)


def test_critical_curve_polyline_distance_matches_pointwise(orc):
    """The vectorised distance (k-d tree on the curve as a polyline, used to
    mask whole images) agrees with the pointwise distance near the curve and
    reports +inf beyond its search radius."""
    r_ = rng(31)
    for a, incl in ((0.9, 80.0), (0.5, 30.0), (0.0, 45.0), (0.998, 5.0)):
        th_o = math.radians(incl)
        al, be = orc.critical_curve_polyline(1.0, a, th_o, 2000)
        # points scattered around the curve and far from it
        k = r_.integers(0, len(al), 200)
        pa = np.concatenate([al[k] + r_.normal(0, 0.08, 200), r_.uniform(-25, 25, 100)])
        pb = np.concatenate([be[k] + r_.normal(0, 0.08, 200), r_.uniform(-25, 25, 100)])
        d_many = orc.critical_curve_distance_many(1.0, a, th_o, pa, pb)
        d_one = np.array([orc.critical_curve_distance(1.0, a, th_o, x, y) for x, y in zip(pa, pb)])
        near = d_one < 0.2
        assert near.sum() > 150
        np.testing.assert_allclose(d_many[near], d_one[near], atol=1e-6)
        assert np.all(np.isinf(d_many[d_one > 0.3]))


def test_drift_flag_marks_rays_whose_norm_the_step_broke(orc):
    """The validity flag: g(u,u) is a constant of the geodesic flow (Sec. 2,
    eq. geo), so an ESCAPED or CAPPED ray whose end norm departs from its
    start norm by more than 1e-3 max(E^2, |g|) is flagged.  On a 96 x 96
    Kerr a = 0.9 camera at 80 degrees traced with h = 0.05 r, the flag is that
    rule exactly, never on CAPTURED or NONFINITE rays; and the same pixels
    traced with a ten times finer step (h = 0.005 r, a reference the coarse
    map approaches as h^4) show that the flag separates the results: escaped
    rays without the flag end within 1e-2 rad of the reference's theta (99% of
    them within 2e-3: the two step rules cross r_esc at different radii, up to
    0.05 r_esc apart, and theta still moves out there), while the flagged ones
    include every ray that ended more than 0.1 rad away."""
    nx = 96
    a, th_o = 0.9, math.radians(80)
    ics = orc.camera_ics(1.0, a, 1000.0, th_o, 25.0, nx, nx, np.arange(nx * nx))
    coarse = orc.trace_many(1.0, a, ics, orc.make_term(0.01, 1100.0, 20_000, 0.0, 0.05))
    fine = orc.trace_many(1.0, a, ics, orc.make_term(0.01, 1100.0, 200_000, 0.0, 0.005))
    f, flag = coarse["fate"] & orc.FATE_MASK, (coarse["fate"] & orc.FATE_DRIFTED) != 0
    n0, n1, E0 = coarse["inv0"][3], coarse["inv1"][3], coarse["inv0"][0]
    rule = np.isin(f, (orc.FATE_ESCAPED, orc.FATE_CAPPED)) & (
        np.abs(n1 - n0) > orc.NORM_DRIFT_TOL * np.maximum(E0 * E0, np.abs(n0)))
    assert np.array_equal(flag, rule)
    assert not flag[np.isin(f, (orc.FATE_CAPTURED, orc.FATE_NONFINITE))].any()
    esc = (f == orc.FATE_ESCAPED) & ((fine["fate"] & orc.FATE_MASK) == orc.FATE_ESCAPED) & \
          ((fine["fate"] & orc.FATE_DRIFTED) == 0)
    err = np.abs(coarse["y"][2] - fine["y"][2])
    good = esc & ~flag
    assert good.sum() > 5000 and flag[esc].sum() > 50
    assert np.all(err[good] < 1e-2) and np.quantile(err[good], 0.99) < 2e-3
    assert np.all(flag[esc & (err > 0.1)])


def test_rhs_noise_option_perturbs_at_the_rounding_level(orc):
    """The oracle's test-only rhs_noise option (a +-delta relative
    perturbation of every right-hand-side component) moves a
    well-conditioned orbit by about delta times the number of evaluations and
    leaves an unperturbed run unchanged: the tool the adaptive-integrator
    parity test uses to measure each ray's sensitivity to rounding."""
    ys = np.stack([orc.circular_state(1.0, 0.5, r, 1) for r in (8.0, 9.0, 11.0)], axis=1)
    ys[5] = 0.01  # eccentric
    for method, extra in ((0, {}), (1, dict(rtol=1e-10, atol=1e-10))):
        t0 = orc.make_term(n_steps_cap=2000, dl=0.05, method=method, **extra)
        t1 = orc.make_term(n_steps_cap=2000, dl=0.05, method=method, rhs_noise=2.0**-52, **extra)
        a, a2 = orc.trace_many(1.0, 0.5, ys, t0), orc.trace_many(1.0, 0.5, ys, t0)
        b = orc.trace_many(1.0, 0.5, ys, t1)
        assert np.array_equal(a["y"], a2["y"])
        rel = np.abs(b["y"] - a["y"]) / np.maximum(np.abs(a["y"]), 1.0)
        assert 0 < rel.max() < 2000 * 8 * 2.0**-52 * 100, rel.max()


# --------------------------------------------------------------------------- generic bound orbits
def test_splitmix64_published_vector(orc):
    """SplitMix64 from state 0: the generator's published first outputs."""
    for k, hx in load_golden("splitmix64_seed0.txt"):
        assert orc.splitmix64(0, int(k)) == int(hx, 16)
    u = [orc.uniform(5, k) for k in range(2000)]
    assert 0 <= min(u) and max(u) < 1 and abs(np.mean(u) - 0.5) < 0.02


def test_bound_orbit_solve_schwarzschild_closed_form(orc):
    """a = 0, equatorial: eccentric Schwarzschild orbits have (textbook, M = 1,
    p = semi-latus rectum) E^2 = ((p-2)^2 - 4e^2)/(p(p-3-e^2)),
    L^2 = p^2/(p-3-e^2)."""
    for rp, e in ((8.0, 0.3), (10.0, 0.6), (7.0, 0.0), (12.0, 0.1)):
        code, E, Lz, Q, r3 = orc.bound_orbit_solve(1.0, 0.0, rp, e, 0.0)
        assert code == 0
        p = rp * (1 + e)
        assert E == pytest.approx(math.sqrt(((p - 2) ** 2 - 4 * e * e) / (p * (p - 3 - e * e))), rel=1e-10)
        assert Lz == pytest.approx(math.sqrt(p * p / (p - 3 - e * e)), rel=1e-10)
        assert Q == pytest.approx(0.0, abs=1e-20)


def test_bound_orbit_solve_kerr_circular_equatorial(orc):
    """e = 0, iota = 0 / pi reduce to Bardeen's prograde / retrograde circular orbits."""
    for a in (0.3, 0.9):
        for r in (10.0, 12.0):  # outside both ISCOs (retrograde ISCO at a = 0.9 is 8.72)
            for iota, pro in ((0.0, 1), (math.pi, 0)):
                code, E, Lz, Q, _ = orc.bound_orbit_solve(1.0, a, r, 0.0, iota)
                Eb, Lb = orc.kerr_circular_bardeen(1.0, a, r, pro)
                assert code == 0
                assert E == pytest.approx(Eb, rel=1e-9) and Lz == pytest.approx(Lb, rel=1e-9)


def test_bound_sampler_properties(orc):
    """Accepted samples: R(rp) = R(ra) = 0, norm = -1, the invariants of the
    state reproduce (E, L_z, Q), cos iota = L_z / sqrt(L_z^2 + Q), the third
    root lies inside rp, and rp lies in [ISCO_pro + 0.5, 10]."""
    seed = 1803083203
    rejected = 0
    for idx in range(300):
        s = orc.bound_sample(1.0, 0.998, seed, idx)
        a = s["a"]
        rp, e, iota, att = s["cand"]
        rejected += int(att) - 1
        if s["accepted"] < 0:
            continue
        code, E, Lz, Q, r3 = orc.bound_orbit_solve(1.0, a, rp, e, iota)
        assert code == 0 and r3 < rp
        E2, Lz2, Q2, norm = orc.invariants(1.0, a, s["y"])
        assert norm == pytest.approx(-1.0, abs=1e-12)
        assert E2 == pytest.approx(E, rel=1e-12) and Lz2 == pytest.approx(Lz, rel=1e-10, abs=1e-12)
        assert Q2 == pytest.approx(Q, rel=1e-9, abs=1e-10)
        assert Lz / math.sqrt(Lz * Lz + Q) == pytest.approx(math.cos(iota), abs=1e-9)
        ra = rp * (1 + e) / (1 - e)
        sc = rp**4
        assert abs(orc.radial_potential(1.0, a, E, Lz, Q, rp)) < 1e-10 * sc
        assert abs(orc.radial_potential(1.0, a, E, Lz, Q, ra)) < 1e-10 * ra**4
        assert orc.isco_bardeen(1.0, a, 1) + 0.5 <= rp <= 10.0
    # plunging candidates exist and are rejected (retrograde near the prograde ISCO)
    assert orc.bound_orbit_solve(1.0, 0.998, 2.0, 0.0, math.pi)[0] != 0
    assert rejected > 0


def test_bound_orbit_conserves_carter_constant(orc):
    """Integrated generic orbits conserve E, L_z, Q and the norm to RK4
    truncation (dtau = 0.02, 5000 steps): relative drift < 1e-8."""
    for idx in range(4):
        s = orc.bound_sample(1.0, 0.998, 1803083203, idx)
        out = orc.trace_one(1.0, s["a"], s["y"], orc.make_term(n_steps_cap=5000, dl=0.02))
        i0 = orc.invariants(1.0, s["a"], s["y"])
        i1 = orc.invariants(1.0, s["a"], out["y"])
        assert np.all(np.abs(i1 - i0) <= 1e-8 * np.maximum(np.abs(i0), 1.0)), (i0, i1)


# --------------------------------------------------------------------------- termination logic
def test_termination_fates_and_step_rule(orc):
    """Captured / non-finite / escaped after each completed step, in that order
    of precedence, capped after the last; h = dl_r_scale * r at the step start;
    lambda is the sum of the steps taken."""
    # radial infall E = 1, L = 0 from r = 10: captured
    y0 = np.zeros(8)
    y0[1], y0[2] = 10.0, math.pi / 2
    y0[4:] = orc.inverse_metric(1.0, 0.0, 10.0, math.pi / 2) @ np.array([-1.0, -math.sqrt(2 / 10) / (1 - 0.2), 0, 0])
    term = orc.make_term(eps_hor=0.01, r_esc=1100.0, n_steps_cap=100_000, dl=0.0, dl_r_scale=0.01)
    out = orc.trace_one(1.0, 0.0, y0, term, stride=1)
    assert out["fate"] == orc.FATE_CAPTURED and out["y"][1] <= 2.02
    tr = out["traj"][: out["steps"] + 1]
    assert out["lambda"] == pytest.approx(np.sum(0.01 * tr[:-1, 1]), rel=1e-13)
    assert np.all(np.isnan(out["traj"][out["steps"] + 1:]))
    # capped
    E, L = orc.schw_circular(1.0, 10.0)
    yc = orc.paper_to_state(1.0, 0.0, [0, 10.0, math.pi / 2, 0, E, 0, 0, L])
    out = orc.trace_one(1.0, 0.0, yc, orc.make_term(n_steps_cap=77, dl=0.01))
    assert out["fate"] == orc.FATE_CAPPED and out["steps"] == 77 and out["lambda"] == pytest.approx(0.77)
    # zero cap: no step
    out = orc.trace_one(1.0, 0.0, yc, orc.make_term(n_steps_cap=0, dl=0.01))
    assert out["fate"] == orc.FATE_CAPPED and out["steps"] == 0 and np.array_equal(out["y"], yc)
    # escaped
    ye = _equatorial_null(orc, 0.0, 50.0, 20.0, inward=False)
    out = orc.trace_one(1.0, 0.0, ye, orc.make_term(r_esc=60.0, n_steps_cap=10_000, dl=0.0, dl_r_scale=0.01))
    assert out["fate"] == orc.FATE_ESCAPED and out["y"][1] >= 60.0
    # non-finite
    yn = yc.copy()
    yn[7] = np.nan
    out = orc.trace_one(1.0, 0.0, yn, orc.make_term(n_steps_cap=10, dl=0.01))
    assert out["fate"] == orc.FATE_NONFINITE and out["steps"] == 1


def test_strided_samples_equal_shorter_runs(orc):
    """Trajectory sample k is the state after k*stride steps (bitwise equal to
    the final state of a run capped there)."""
    s = orc.bound_sample(1.0, 0.9, 11, 3)
    term = orc.make_term(n_steps_cap=100, dl=0.05)
    tr = orc.trace_one(1.0, s["a"], s["y"], term, stride=25)["traj"]
    assert tr.shape == (5, 8)
    for k in range(5):
        y = orc.trace_one(1.0, s["a"], s["y"], orc.make_term(n_steps_cap=25 * k, dl=0.05))["y"]
        assert np.array_equal(tr[k], y)


def test_trace_many_matches_trace_one(orc):
    """The multi-ray (OpenMP) loop gives the same bits as ray-by-ray calls and
    per-ray spins are honoured."""
    n = 37
    ys, spins, _ = orc.bound_samples(1.0, 0.998, 5, np.arange(n))
    term = orc.make_term(n_steps_cap=300, dl=0.02)
    many = orc.trace_many(1.0, 0.0, ys, term, a_per_ray=spins, nthreads=4)
    for i in range(n):
        one = orc.trace_one(1.0, spins[i], ys[:, i], term)
        assert np.array_equal(many["y"][:, i], one["y"])
        assert many["steps"][i] == one["steps"] and many["fate"][i] == one["fate"]
        np.testing.assert_array_equal(many["inv0"][:, i], orc.invariants(1.0, spins[i], ys[:, i]))


# --------------------------------------------------------------------------- canonical form (eq. Ham)
def test_canonical_trace_conserves_E_and_Lz_exactly(orc):
    """Sec. 2 eq. Ham: H does not depend on t or phi, so p_t = -E and p_phi =
    L_z never change along the canonical RK4 trace; the only error left in E
    and L_z is the conversion (x, u) <-> (x, p) at the two ends, while the
    geodesic form drifts by the RK4 truncation error."""
    ys, spins, _ = orc.bound_samples(1.0, 0.9, 11, np.arange(24), spin_fixed=True)
    geo = orc.make_term(n_steps_cap=4000, dl=0.25)
    can = orc.make_term(n_steps_cap=4000, dl=0.25, form=1)
    worst_can, worst_geo = 0.0, 0.0
    for i in range(ys.shape[1]):
        i0 = orc.invariants(1.0, 0.9, ys[:, i])
        a = orc.trace_one(1.0, 0.9, ys[:, i], geo)
        b = orc.trace_one(1.0, 0.9, ys[:, i], can)
        if a["fate"] != 3 or b["fate"] != 3:
            continue
        ig, ic = orc.invariants(1.0, 0.9, a["y"]), orc.invariants(1.0, 0.9, b["y"])
        worst_geo = max(worst_geo, np.abs(ig[:2] - i0[:2]).max())
        worst_can = max(worst_can, np.abs(ic[:2] - i0[:2]).max())
    assert worst_can < 1e-12
    assert worst_geo > 1e3 * worst_can


def test_canonical_and_geodesic_forms_agree_to_fourth_order(orc):
    """The two forms are exact rewritings of one flow; their RK4 maps differ by
    the truncation error, which falls as h^4 (ratio 16 when h halves)."""
    y0 = orc.circular_state(1.0, 0.6, 9.0, 1)
    y0[5] = 0.05  # perturb into an eccentric, inclined orbit
    y0[6] = 0.01
    diffs = []
    for h in (0.4, 0.2, 0.1):
        n = int(round(200.0 / h))
        a = orc.trace_one(1.0, 0.6, y0, orc.make_term(n_steps_cap=n, dl=h))
        b = orc.trace_one(1.0, 0.6, y0, orc.make_term(n_steps_cap=n, dl=h, form=1))
        diffs.append(np.abs(a["y"] - b["y"]).max())
    assert 12.0 < diffs[0] / diffs[1] < 20.0 and 12.0 < diffs[1] / diffs[2] < 20.0, diffs


def test_canonical_circular_orbit_stays_closed(orc):
    """Sec. 4 circular orbits in the canonical form: r stays at r0 and phi
    advances at the analytic angular frequency (eq. omega), as in the geodesic
    form."""
    for a, r0 in ((0.0, 8.0), (0.7, 7.0)):
        y0 = orc.circular_state(1.0, a, r0, 1)
        t = orc.make_term(n_steps_cap=5000, dl=0.02, form=1)
        res = orc.trace_one(1.0, a, y0, t)
        assert abs(res["y"][1] - r0) < 1e-9
        om = y0[7] / y0[4]
        assert res["y"][3] == pytest.approx(om * res["y"][0], rel=1e-10)


# --------------------------------------------------------------------------- 3+1 form (eq. ADM)
def _fd4(f, x, h):
    """Fourth-order central difference of f at x."""
    return (-f(x + 2 * h) + 8 * f(x + h) - 8 * f(x - h) + f(x - 2 * h)) / (12 * h)


def test_adm_derivatives_match_finite_differences(orc):
    """Sec. 2: the r- and theta-derivatives of Kerr's lapse, shift and
    3-metric (the expressions after eq. coord) against fourth-order finite
    differences of the values themselves."""
    r_ = rng(21)
    for _ in range(40):
        a = r_.uniform(0.0, 0.999)
        r = r_.uniform(2.2, 40.0)
        th = r_.uniform(0.1, math.pi - 0.1)
        da, db, dg = orc.adm_derivs(M1, a, r, th)

        def vals(rr, tt):
            al, be, ga = orc.adm(M1, a, rr, tt)
            return np.concatenate([[al, be], ga])

        fr = _fd4(lambda x: vals(x, th), r, 1e-3 * r)
        ft = _fd4(lambda x: vals(r, x), th, 1e-3)
        got_r = np.concatenate([[da[0], db[0]], dg[:, 0]])
        got_t = np.concatenate([[da[1], db[1]], dg[:, 1]])
        scale_r = np.abs(vals(r, th)) / r + 1e-12
        scale_t = np.abs(vals(r, th)) + 1e-12
        assert np.all(np.abs(got_r - fr) < 1e-7 * scale_r), (got_r, fr)
        assert np.all(np.abs(got_t - ft) < 1e-7 * scale_t), (got_t, ft)


def test_adm_assembled_metric_is_kerr(orc):
    """Eq. ADM assembled from alpha, beta^i, gamma_ij (full sums over i, j)
    reproduces eq. kerr and its analytic derivatives, which have their own
    pins above."""
    r_ = rng(22)
    for _ in range(40):
        a = r_.uniform(0.0, 0.999)
        r = r_.uniform(2.2, 60.0)
        th = r_.uniform(0.05, math.pi - 0.05)
        g, ga = orc.metric(M1, a, r, th), orc.adm_metric(M1, a, r, th)
        np.testing.assert_allclose(ga, g, rtol=1e-12, atol=1e-14 * np.abs(g).max())
        d, dga = orc.metric_derivs(M1, a, r, th), orc.adm_metric_derivs(M1, a, r, th)
        np.testing.assert_allclose(dga, d, rtol=1e-10, atol=1e-12 * np.abs(d).max())


def test_invert4_matches_library_inverse(orc):
    """The oracle's Gauss-Jordan inverse against numpy's LAPACK inverse, on
    random matrices and on Kerr metrics (indefinite, with a zero pivot in
    the unpivoted order at a = 0)."""
    r_ = rng(23)
    for _ in range(50):
        A = r_.normal(size=(4, 4)) + 3 * np.eye(4)
        np.testing.assert_allclose(orc.invert4(A), np.linalg.inv(A), rtol=1e-10, atol=1e-12)
    for a in (0.0, 0.5, 0.99):
        g = orc.metric(M1, a, 6.0, 1.1)
        np.testing.assert_allclose(orc.invert4(g) @ g, np.eye(4), atol=1e-13)
        np.testing.assert_allclose(orc.invert4(g), orc.inverse_metric(M1, a, 6.0, 1.1), rtol=1e-12, atol=1e-15)


def _random_canonical(r_, a):
    y = _random_state(r_, a)
    return np.concatenate([y[:4], orc_momenta(a, y)]), y


def orc_momenta(a, y):
    import oracle

    return oracle.state_to_momenta(M1, a, y)


def test_adm_rhs_is_hamiltons_equations(orc):
    """Sec. 2 eq. Ham taken literally: dx^mu/dl = dH/dp_mu and dp_mu/dl =
    -dH/dx^mu, with H = g^{mn} p_m p_n / 2 differentiated numerically, match
    the 3+1 right-hand side; and H at p = g u equals g(u, u) / 2."""
    r_ = rng(24)
    for _ in range(30):
        a = r_.uniform(0.0, 0.999)
        z, y = _random_canonical(r_, a)
        f = orc.rhs_adm(M1, a, z)
        g = orc.metric(M1, a, y[1], y[2])
        assert orc.hamiltonian_adm(M1, a, z) == pytest.approx(0.5 * y[4:] @ g @ y[4:], rel=1e-10, abs=1e-12)
        grad = np.zeros(8)
        for k in range(8):
            e = np.zeros(8)
            hk = 1e-4 * max(1.0, abs(z[k]))
            e[k] = 1.0
            grad[k] = _fd4(lambda s: orc.hamiltonian_adm(M1, a, z + s * e), 0.0, hk)
        np.testing.assert_allclose(f[:4], grad[4:], rtol=1e-7, atol=1e-9 * np.abs(grad[4:]).max())
        np.testing.assert_allclose(f[4:], -grad[:4], rtol=1e-6, atol=1e-8 * np.abs(grad[:4]).max() + 1e-12)
        assert f[4] == 0.0 and f[7] == 0.0


def test_adm_rhs_equals_kerr_canonical_rhs(orc):
    """The 3+1 route (g assembled from alpha, beta, gamma, numerically inverted)
    and the BL route (closed-form inverse of eq. kerr) are the same equations."""
    r_ = rng(25)
    for _ in range(60):
        a = r_.uniform(0.0, 0.999)
        z, _ = _random_canonical(r_, a)
        fa, fh = orc.rhs_adm(M1, a, z), orc.rhs_hamiltonian(M1, a, z)
        np.testing.assert_allclose(fa, fh, rtol=1e-10, atol=1e-12 * np.abs(fh).max())


def test_adm_trace_matches_canonical_and_conserves(orc):
    """Form 2 (eq. Ham with g from eq. ADM) is the same discrete RK4 map as
    form 1 up to rounding: traces agree closely, p_t and p_phi are exact
    constants, and a circular orbit stays at r0 with phi advancing at eq.
    omega's rate."""
    ys, spins, _ = orc.bound_samples(1.0, 0.9, 11, np.arange(12), spin_fixed=True)
    can = orc.make_term(n_steps_cap=3000, dl=0.25, form=1)
    adm = orc.make_term(n_steps_cap=3000, dl=0.25, form=2)
    for i in range(ys.shape[1]):
        i0 = orc.invariants(1.0, 0.9, ys[:, i])
        a = orc.trace_one(1.0, 0.9, ys[:, i], can)
        b = orc.trace_one(1.0, 0.9, ys[:, i], adm)
        assert a["fate"] == b["fate"] and a["steps"] == b["steps"]
        scale = np.maximum(np.abs(a["y"]), 1.0)
        assert np.all(np.abs(a["y"] - b["y"]) < 1e-7 * scale), (a["y"], b["y"])
        if b["fate"] == 3:
            assert np.abs(orc.invariants(1.0, 0.9, b["y"])[:2] - i0[:2]).max() < 1e-12
    for a, r0 in ((0.0, 8.0), (0.7, 7.0)):
        y0 = orc.circular_state(1.0, a, r0, 1)
        res = orc.trace_one(1.0, a, y0, orc.make_term(n_steps_cap=5000, dl=0.02, form=2))
        assert abs(res["y"][1] - r0) < 1e-9
        assert res["y"][3] == pytest.approx(y0[7] / y0[4] * res["y"][0], rel=1e-10)


# --------------------------------------------------------------------------- Dormand-Prince 5(4)
def _rk_order_conditions(b, A, c, order):
    """Residuals of the Runge-Kutta order conditions (Butcher trees) up to
    `order` (at most 5) for weights b, matrix A, nodes c."""
    one = np.ones_like(c)
    Ac = A @ c
    res = [b @ one - 1.0]
    if order >= 2:
        res += [b @ c - 1 / 2]
    if order >= 3:
        res += [b @ c**2 - 1 / 3, b @ Ac - 1 / 6]
    if order >= 4:
        res += [b @ c**3 - 1 / 4, b @ (c * Ac) - 1 / 8, b @ (A @ c**2) - 1 / 12, b @ (A @ Ac) - 1 / 24]
    if order >= 5:
        res += [b @ c**4 - 1 / 5, b @ (c**2 * Ac) - 1 / 10, b @ (c * (A @ c**2)) - 1 / 15,
                b @ (c * (A @ Ac)) - 1 / 30, b @ (Ac * Ac) - 1 / 20, b @ (A @ c**3) - 1 / 20,
                b @ (A @ (c * Ac)) - 1 / 40, b @ (A @ (A @ c**2)) - 1 / 60, b @ (A @ (A @ Ac)) - 1 / 120]
    return np.array(res)


def test_dopri5_tableau_satisfies_order_conditions(orc):
    """The typed Dormand-Prince coefficients against the theory they must
    satisfy: row sums equal the nodes, the fifth-order weights meet all 17
    conditions to order 5, the embedded weights all 8 to order 4 but not all
    of order 5, and the last stage is the fifth-order result (FSAL)."""
    c, A, b, bh = orc.dopri5_tableau()
    np.testing.assert_allclose(A.sum(axis=1), c, atol=1e-15)
    assert np.all(np.triu(A) == 0.0)
    assert np.abs(_rk_order_conditions(b, A, c, 5)).max() < 1e-15
    assert np.abs(_rk_order_conditions(bh, A, c, 4)).max() < 1e-15
    assert np.abs(_rk_order_conditions(bh, A, c, 5)[8:]).max() > 1e-5
    np.testing.assert_array_equal(A[6], b)


def test_dopri5_linear_step_is_its_stability_polynomial(orc):
    """On y' = lam y one Dormand-Prince step multiplies y by the stability
    function R(z) = sum_{k<=5} z^k/k! + z^6/600 (Hairer & Wanner, Solving
    ODEs II, Sec. IV.2), and its error estimate falls as h^5."""
    for z in (-0.5, -0.1, 0.05, 0.3, -2.0):
        y5, _ = orc.dopri5_linear(z, 1.0, 1.0)
        R = sum(z**k / math.factorial(k) for k in range(6)) + z**6 / 600
        assert y5 == pytest.approx(R, rel=1e-14, abs=1e-16)
    e1 = abs(orc.dopri5_linear(-1.0, 0.1, 1.0)[1])
    e2 = abs(orc.dopri5_linear(-1.0, 0.05, 1.0)[1])
    assert 28.0 < e1 / e2 < 36.0


def test_dopri5_trace_meets_tolerance(orc):
    """Adaptive traces of generic bound Kerr orbits (3000 attempts): E, L_z,
    Q and the norm, exact invariants of the flow, drift by less than the
    attempts times the tolerance, ten times less at tolerance 1e-12 than at
    1e-10, and the tighter tolerance covers less lambda in as many attempts; a circular orbit stays at r0 with phi advancing at the
    angular frequency of eq. omega."""
    ys, spins, _ = orc.bound_samples(1.0, 0.9, 11, np.arange(8), spin_fixed=True)
    drift, rate = {}, {}
    for tol in (1e-10, 1e-12):
        t = orc.make_term(n_steps_cap=3000, dl=0.01, method=1, rtol=tol, atol=tol)
        d_max, lam_sum = 0.0, 0.0
        for i in range(ys.shape[1]):
            got = orc.trace_one(1.0, 0.9, ys[:, i], t)
            assert got["fate"] == 3 and got["steps"] == 3000
            i0, i1 = orc.invariants(1.0, 0.9, ys[:, i]), orc.invariants(1.0, 0.9, got["y"])
            d_max = max(d_max, (np.abs(i1 - i0) / np.maximum(np.abs(i0), 1.0)).max())
            lam_sum += got["lambda"]
        drift[tol], rate[tol] = d_max, lam_sum
    # the local error per accepted step is held below tol (times the scale
    # of the state); over 3000 attempts the drift stays below 3000 tol
    assert drift[1e-10] < 3000 * 1e-10 and drift[1e-12] < 3000 * 1e-12, drift
    assert drift[1e-12] < drift[1e-10] / 10, drift
    assert rate[1e-12] < rate[1e-10], rate
    y0 = orc.circular_state(1.0, 0.7, 7.0, 1)
    res = orc.trace_one(1.0, 0.7, y0, orc.make_term(n_steps_cap=3000, dl=0.1, method=1, rtol=1e-11, atol=1e-11))
    assert res["fate"] == 3 and abs(res["y"][1] - 7.0) < 1e-8
    assert res["y"][3] == pytest.approx(y0[7] / y0[4] * res["y"][0], rel=1e-8)


def test_dopri5_step_control_and_capture(orc):
    """The controller grows a tiny first step (far fewer attempts than
    lambda / dl), caps steps at dl_r_scale r, and a radially infalling ray is
    captured as with RK4."""
    y0 = orc.circular_state(1.0, 0.0, 10.0, 1)
    res = orc.trace_one(1.0, 0.0, y0, orc.make_term(n_steps_cap=500, dl=1e-6, method=1, rtol=1e-9, atol=1e-9))
    assert res["lambda"] > 1e3 * 1e-6 * res["steps"]
    capped = orc.trace_one(1.0, 0.0, y0, orc.make_term(n_steps_cap=200, dl=1e-6, dl_r_scale=0.01, method=1,
                                                        rtol=1e-6, atol=1e-6))
    assert capped["lambda"] <= 0.01 * 10.0 * 200 * (1 + 1e-12)
    # radial infall from rest at r = 10 (Schwarzschild): u^t = 1/sqrt(1 - 2/10)
    yi = np.array([0.0, 10.0, math.pi / 2, 0.0, 1.0 / math.sqrt(0.8), 0.0, 0.0, 0.0])
    a = orc.trace_one(1.0, 0.0, yi, orc.make_term(n_steps_cap=10000, dl=0.01, method=1, rtol=1e-9, atol=1e-9))
    b = orc.trace_one(1.0, 0.0, yi, orc.make_term(n_steps_cap=10000, dl=0.01))
    assert a["fate"] == b["fate"] == 1


def test_dopri5_canonical_forms_keep_pt_pphi_and_follow_the_flow(orc):
    """Dormand-Prince in the canonical forms (eq. Ham through eq. kerr, and
    through eq. ADM): p_t and p_phi have zero derivative, so E and L_z come
    back to the conversions' rounding; Q and the norm drift within attempts x
    tol, as in the geodesic form."""
    ys, spins, _ = orc.bound_samples(1.0, 0.9, 13, np.arange(6), spin_fixed=True)
    for form in (1, 2):
        t = orc.make_term(n_steps_cap=800, dl=0.02, form=form, method=1, rtol=1e-10, atol=1e-10)
        for i in range(ys.shape[1]):
            res = orc.trace_one(1.0, 0.9, ys[:, i], t)
            assert res["fate"] == 3
            i0, i1 = orc.invariants(1.0, 0.9, ys[:, i]), orc.invariants(1.0, 0.9, res["y"])
            d = np.abs(i1 - i0) / np.maximum(np.abs(i0), 1.0)
            assert d[:2].max() < 1e-12, (form, d)
            assert d[2:].max() < 800 * 1e-10, (form, d)


def test_kerr_equatorial_escape_angle_matches_quadrature(orc):
    """The final phi of escaped null rays, pinned directly [not in paper]:
    for a Kerr (a = 0.9) equatorial ray from r = 1000M with E = 1 and L = b
    (Q = 0), Bardeen's first integrals give dphi/dr = (L - aE + aP/Delta) /
    sqrt(R) with P = E(r^2 + a^2) - aL and R = P^2 - Delta (L - aE)^2, so the
    angle swept in to the periapsis r_p (the largest root of R) and out to
    the final radius is a quadrature (r = r_p + u^2 removes the square-root
    end point).  The oracle's trace with fine steps (h = 5e-4 r) ends at that
    angle within 1e-9 for prograde, retrograde and wide rays, and theta stays
    pi/2."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    M, a, r_obs, E = 1.0, 0.9, 1000.0, 1.0
    for b in (6.0, 10.0, -8.0, 25.0):
        L = b
        Delta = lambda r: r * r - 2 * M * r + a * a  # noqa: E731
        P = lambda r: E * (r * r + a * a) - a * L  # noqa: E731
        R = lambda r: P(r) ** 2 - Delta(r) * (L - a * E) ** 2  # noqa: E731
        grid = np.linspace(1.5, 50.0, 20000)
        vals = np.array([R(x) for x in grid])
        k = np.where((vals[:-1] < 0) & (vals[1:] >= 0))[0][-1]
        rp = brentq(R, grid[k], grid[k + 1], xtol=1e-15)

        def leg(r1):
            f = lambda u: 2 * u * (L - a * E + a * P(rp + u * u) / Delta(rp + u * u)) / math.sqrt(  # noqa: E731
                max(R(rp + u * u), 1e-300))
            return quad(f, 0.0, math.sqrt(r1 - rp), epsabs=1e-13, epsrel=1e-13, limit=500)[0]

        gi = orc.inverse_metric(M, a, r_obs, math.pi / 2)
        p = np.array([-E, -math.sqrt(R(r_obs)) / Delta(r_obs), 0.0, L])
        y0 = np.concatenate([[0.0, r_obs, math.pi / 2, 0.0], gi @ p])
        res = orc.trace_one(M, a, y0, orc.make_term(0.01, 1100.0, 10**6, 0.0, 5e-4))
        assert res["fate"] == orc.FATE_ESCAPED
        assert res["y"][2] == math.pi / 2
        assert abs(res["y"][3] - (leg(r_obs) + leg(res["y"][1]))) < 1e-9, b


def test_kerr_escape_angles_match_mino_time_integrals(orc):
    """The final (theta, phi) of escaped off-equatorial null rays, pinned
    directly [not in paper]: in Mino time (dl = rho^2 dl_M) Kerr null
    geodesics obey dr/dl_M = +-sqrt(R(r)), du/dl_M = -+sqrt(a^2 (u+^2 - u^2)
    (u^2 + u-^2)) with u = cos(theta), and dphi/dl_M = aP/Delta + L/(1 - u^2)
    - aE.  The Mino time spent on the radial path (in to the periapsis, out to
    the final radius) fixes where u is on its oscillation between -u+ and u+
    (with u = u+ sin(psi) the oscillation's time is the smooth integral of
    1 / (a sqrt(u+^2 sin^2 psi + u-^2))), and phi is the r-part integrated
    along the radial path plus the u-part integrated along that oscillation.
    The oracle's trace (h = 5e-4 r) ends at the predicted angles within 1e-9,
    for both initial directions of theta and two inclinations (a = 0.9,
    E = 1)."""
    from scipy.integrate import quad
    from scipy.optimize import brentq

    M, a, r_obs, E = 1.0, 0.9, 1000.0, 1.0
    for L, Q, th0, sgn in ((3.0, 20.0, math.radians(80), 1), (-5.0, 30.0, math.radians(80), -1),
                           (8.0, 50.0, math.radians(60), 1), (2.0, 60.0, math.radians(80), -1)):
        Delta = lambda r: r * r - 2 * M * r + a * a  # noqa: E731
        P = lambda r: E * (r * r + a * a) - a * L  # noqa: E731
        R = lambda r: P(r) ** 2 - Delta(r) * ((L - a * E) ** 2 + Q)  # noqa: E731
        grid = np.linspace(1.5, 60.0, 40000)
        vals = np.array([R(x) for x in grid])
        k = np.where((vals[:-1] < 0) & (vals[1:] >= 0))[0][-1]
        rp = brentq(R, grid[k], grid[k + 1], xtol=1e-15)

        def leg(r1, g=lambda r: 1.0):
            f = lambda v: 2 * v * g(rp + v * v) / math.sqrt(max(R(rp + v * v), 1e-300))  # noqa: E731
            return quad(f, 0.0, math.sqrt(r1 - rp), epsabs=1e-14, epsrel=1e-14, limit=500)[0]

        A, B = a * a, Q + L * L - a * a
        up2 = (-B + math.sqrt(B * B + 4 * A * Q)) / (2 * A)
        um2 = (B + math.sqrt(B * B + 4 * A * Q)) / (2 * A)
        up = math.sqrt(up2)
        w = lambda x: 1.0 / (a * math.sqrt(up2 * math.sin(x) ** 2 + um2))  # noqa: E731

        def Phi(psi):
            return quad(w, 0.0, psi, epsabs=1e-14, epsrel=1e-14)[0]

        def Jphi(p1, p2):
            f = lambda x: (L / (1.0 - up2 * math.sin(x) ** 2) - a * E) * w(x)  # noqa: E731
            return quad(f, p1, p2, epsabs=1e-13, epsrel=1e-13, limit=200)[0]

        half = Phi(math.pi / 2)

        def psi_of(target):
            if target >= half:
                return math.pi / 2
            if target <= -half:
                return -math.pi / 2
            return brentq(lambda x: Phi(x) - target, -math.pi / 2, math.pi / 2, xtol=1e-15)

        Theta = Q + a * a * E * E * math.cos(th0) ** 2 - L * L / math.tan(th0) ** 2
        gi = orc.inverse_metric(M, a, r_obs, th0)
        p = np.array([-E, -math.sqrt(R(r_obs)) / Delta(r_obs), sgn * math.sqrt(Theta), L])
        y0 = np.concatenate([[0.0, r_obs, th0, 0.0], gi @ p])
        res = orc.trace_one(M, a, y0, orc.make_term(0.01, 1100.0, 10**6, 0.0, 5e-4))
        assert res["fate"] == orc.FATE_ESCAPED
        rf = res["y"][1]
        G = leg(r_obs) + leg(rf)
        phi = leg(r_obs, lambda r: a * P(r) / Delta(r)) + leg(rf, lambda r: a * P(r) / Delta(r))
        # phase on the oscillation: [0, 2 half) u falling from u+, [2 half, 4 half) rising from -u+
        psi0 = math.asin(math.cos(th0) / up)
        s = half - Phi(psi0) if sgn > 0 else 3 * half + Phi(psi0)
        rem = G
        while rem > 0:
            sm = s % (4 * half)
            falling = sm < 2 * half
            psi_now = psi_of(half - sm if falling else sm - 3 * half)
            step = min(rem, (2 * half - sm) if falling else (4 * half - sm))
            sm2 = sm + step
            psi_next = psi_of(half - sm2 if falling else sm2 - 3 * half)
            phi += Jphi(min(psi_now, psi_next), max(psi_now, psi_next))
            rem -= step
            s += step
        assert abs(res["y"][2] - math.acos(up * math.sin(psi_next))) < 1e-9, (L, Q)
        assert abs(res["y"][3] - phi) < 1e-9, (L, Q)


def test_eccentric_equatorial_kerr_orbit_radial_period(orc):
    """Bound timelike Kerr dynamics pinned directly [not in paper]: for an
    eccentric equatorial orbit (periapsis r_p, apoapsis r_a, E and L_z from
    R(r_p) = R(r_a) = 0) Bardeen's first integrals give the proper time of one
    radial period, T_r = 2 int r^2 / sqrt(R) dr, and the advances of phi and t
    over it, 2 int (aP/Delta - aE + L) / sqrt(R) dr and 2 int ((r^2 + a^2)
    P/Delta - a(aE - L)) / sqrt(R) dr (R = (1 - E^2) r (r_a - r)(r - r_p)(r -
    r_3) for Q = 0; r = (r_p + r_a)/2 - (r_a - r_p)/2 cos(chi) makes the
    integrands smooth).  Started at r_p and traced for exactly T_r (40000
    steps), the oracle is back at r_p within 1e-10 with phi and t within 1e-9
    of the quadratures."""
    from scipy.integrate import quad

    M = 1.0
    for a, rp, ra in ((0.9, 8.0, 14.0), (0.5, 7.0, 20.0), (0.9, 10.0, 11.0)):
        code, E, L, Q, r3 = orc.bound_orbit_solve(M, a, rp, (ra - rp) / (ra + rp), 0.0)
        assert code == 0 and Q == 0.0
        Delta = lambda r: r * r - 2 * M * r + a * a  # noqa: E731
        P = lambda r: E * (r * r + a * a) - a * L  # noqa: E731
        rm, rh = 0.5 * (rp + ra), 0.5 * (ra - rp)
        r_of = lambda x: rm - rh * math.cos(x)  # noqa: E731
        den = lambda r: math.sqrt((1 - E * E) * r * (r - r3))  # noqa: E731

        def period_integral(g):
            return 2 * quad(lambda x: g(r_of(x)) / den(r_of(x)), 0.0, math.pi, epsabs=1e-13, epsrel=1e-13)[0]

        Tr = period_integral(lambda r: r * r)
        dphi = period_integral(lambda r: a * P(r) / Delta(r) - a * E + L)
        dt = period_integral(lambda r: (r * r + a * a) * P(r) / Delta(r) - a * (a * E - L))
        gi = orc.inverse_metric(M, a, rp, math.pi / 2)
        y0 = np.concatenate([[0.0, rp, math.pi / 2, 0.0], gi @ np.array([-E, 0.0, 0.0, L])])
        res = orc.trace_one(M, a, y0, orc.make_term(0.01, 1e9, 40000, Tr / 40000, 0.0))
        assert res["fate"] == orc.FATE_CAPPED
        assert abs(res["y"][1] - rp) < 1e-10, (a, rp, ra)
        assert abs(res["y"][3] - dphi) < 1e-9, (a, rp, ra)
        assert abs(res["y"][0] - dt) < 1e-9 * dt, (a, rp, ra)

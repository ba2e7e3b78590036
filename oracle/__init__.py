"""FP64 CPU oracle for Boyer-Lindquist Kerr/Schwarzschild geodesics (RK4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product (the
CUDA library and its binding) never imports it, and it imports nothing from the
product.  The arithmetic lives in ``oracle.c`` (plain C, double precision);
this module only builds it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

FATE_CAPTURED, FATE_ESCAPED, FATE_CAPPED, FATE_NONFINITE = 1, 2, 3, 4
FATE_DRIFTED, FATE_MASK, NORM_DRIFT_TOL = 0x80, 0x7F, 1e-3  # validity flag or-ed into a fate

_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32


class Term(ctypes.Structure):
    """Termination / step rule (mirrors orc_term)."""

    _fields_ = [
        ("eps_hor", _D),
        ("r_esc", _D),
        ("n_steps_cap", _U32),
        ("dl", _D),
        ("dl_r_scale", _D),
        ("form", _U32),
        ("method", _U32),
        ("rtol", _D),
        ("atol", _D),
        ("rhs_noise", _D),
    ]


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, no fast-math, no
    FMA contraction, OpenMP for the timed multi-ray loop)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-std=gnu11",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    def sig(name, res, *args):
        f = getattr(L, name)
        f.restype = res
        f.argtypes = list(args)

    sig("orc_r_plus", _D, _D, _D)
    for n in ("orc_metric", "orc_inverse_metric"):
        sig(n, None, _D, _D, _D, _D, _PD)
    sig("orc_metric_derivs", None, _D, _D, _D, _D, _PD)
    sig("orc_christoffel", None, _D, _D, _D, _D, _PD)
    sig("orc_adm", None, _D, _D, _D, _D, _PD, _PD, _PD)
    sig("orc_rhs", None, _D, _D, _PD, _PD)
    sig("orc_rhs_hamiltonian", None, _D, _D, _PD, _PD)
    sig("orc_adm_derivs", None, _D, _D, _D, _D, _PD, _PD, _PD)
    sig("orc_adm_metric", None, _D, _D, _D, _D, _PD)
    sig("orc_adm_metric_derivs", None, _D, _D, _D, _D, _PD)
    sig("orc_invert4", None, _PD, _PD)
    sig("orc_rhs_adm", None, _D, _D, _PD, _PD)
    sig("orc_hamiltonian_adm", _D, _D, _D, _PD)
    sig("orc_rk4_step_adm", None, _D, _D, _D, _PD)
    sig("orc_dopri5_tableau", None, _PD, _PD, _PD, _PD)
    sig("orc_dopri5_linear_test", None, _D, _D, _D, _PD, _PD)
    sig("orc_rk4_linear_test", None, _D, _D, ctypes.c_int, _PD)
    sig("orc_rk4_step", None, _D, _D, _D, _PD)
    sig("orc_rk4_step_hamiltonian", None, _D, _D, _D, _PD)
    sig("orc_trace_one", ctypes.c_int, _D, _D, _PD, ctypes.POINTER(Term), _PD, _PD,
        ctypes.POINTER(_U32), _PD, _U32)
    sig("orc_trace_many", ctypes.c_int, _D, _D, ctypes.c_void_p, _PD, _U64, ctypes.POINTER(Term),
        _PD, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, _U32, ctypes.c_int)
    sig("orc_invariants", None, _D, _D, _PD, _PD)
    sig("orc_paper_to_state", None, _D, _D, _PD, _PD)
    sig("orc_state_to_momenta", None, _D, _D, _PD, _PD)
    sig("orc_bl_to_cartesian", None, _D, _D, _D, _D, _PD)
    sig("orc_schw_circular", None, _D, _D, _PD, _PD)
    sig("orc_schw_gralorbits", None, _D, _D, _PD, _PD)
    sig("orc_kerr_circular_paper", None, _D, _D, _D, ctypes.c_int, _PD, _PD)
    sig("orc_kerr_circular_bardeen", None, _D, _D, _D, ctypes.c_int, _PD, _PD)
    sig("orc_kerr_omega", _D, _D, _D, _D, _D, _D)
    sig("orc_isco_bardeen", _D, _D, _D, ctypes.c_int)
    sig("orc_isco_paper_literal", _D, _D, _D, ctypes.c_int)
    sig("orc_dEdr_numeric_root", _D, _D, _D, ctypes.c_int, _D, _D)
    sig("orc_photon_orbit", _D, _D, _D, ctypes.c_int)
    sig("orc_circular_state", None, _D, _D, _D, ctypes.c_int, _PD)
    sig("orc_camera_ic", None, _D, _D, _D, _D, _D, _U32, _U32, _U64, _PD)
    sig("orc_critical_curve_distance", _D, _D, _D, _D, _D, _D)
    sig("orc_critical_curve_polyline", None, _D, _D, _D, ctypes.c_int, _PD, _PD)
    sig("orc_splitmix64", _U64, _U64, _U64)
    sig("orc_uniform", _D, _U64, _U64)
    sig("orc_bound_orbit_solve", ctypes.c_int, _D, _D, _D, _D, _D, _PD, _PD, _PD, _PD)
    sig("orc_bound_sample", ctypes.c_int, _D, _D, ctypes.c_int, _U64, _U64, _PD, _PD, _PD)
    sig("orc_radial_potential", _D, _D, _D, _D, _D, _D, _D)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_PD)


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def make_term(eps_hor=0.01, r_esc=1e30, n_steps_cap=1000, dl=0.01, dl_r_scale=0.0, form=0, method=0, rtol=0.0,
              atol=0.0, rhs_noise=0.0) -> Term:
    """form 0: geodesic equation (eq. geo); 1: canonical equations (eq. Ham)
    with g of eq. kerr; 2: the same equations with g from eq. ADM.  method 0:
    classical RK4; 1: Dormand-Prince 5(4) with step-size control (rtol, atol).
    rhs_noise (tests only): relative +- perturbation of every right-hand-side
    component, to measure a ray's sensitivity to rounding."""
    return Term(float(eps_hor), float(r_esc), int(n_steps_cap), float(dl), float(dl_r_scale), int(form),
                int(method), float(rtol), float(atol), float(rhs_noise))


# ---------------------------------------------------------------- geometry
def r_plus(M, a):
    return lib().orc_r_plus(M, a)


def metric(M, a, r, th):
    g = np.zeros(16)
    lib().orc_metric(M, a, r, th, _p(g))
    return g.reshape(4, 4)


def inverse_metric(M, a, r, th):
    g = np.zeros(16)
    lib().orc_inverse_metric(M, a, r, th, _p(g))
    return g.reshape(4, 4)


def metric_derivs(M, a, r, th):
    d = np.zeros(64)
    lib().orc_metric_derivs(M, a, r, th, _p(d))
    return d.reshape(4, 4, 4)


def christoffel(M, a, r, th):
    G = np.zeros(64)
    lib().orc_christoffel(M, a, r, th, _p(G))
    return G.reshape(4, 4, 4)


def adm(M, a, r, th):
    al, be = _D(), _D()
    ga = np.zeros(3)
    lib().orc_adm(M, a, r, th, ctypes.byref(al), ctypes.byref(be), _p(ga))
    return al.value, be.value, ga


def adm_derivs(M, a, r, th):
    """(d alpha, d beta^phi, d gamma_ii) along (r, theta): shapes (2,), (2,), (3, 2)."""
    da, db, dg = np.zeros(2), np.zeros(2), np.zeros(6)
    lib().orc_adm_derivs(M, a, r, th, _p(da), _p(db), _p(dg))
    return da, db, dg.reshape(3, 2)


def adm_metric(M, a, r, th):
    g = np.zeros(16)
    lib().orc_adm_metric(M, a, r, th, _p(g))
    return g.reshape(4, 4)


def adm_metric_derivs(M, a, r, th):
    d = np.zeros(64)
    lib().orc_adm_metric_derivs(M, a, r, th, _p(d))
    return d.reshape(4, 4, 4)


def invert4(A):
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(16)
    Ai = np.zeros(16)
    lib().orc_invert4(_p(A), _p(Ai))
    return Ai.reshape(4, 4)


# ---------------------------------------------------------------- dynamics
def rhs(M, a, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    f = np.zeros(8)
    lib().orc_rhs(M, a, _p(y), _p(f))
    return f


def rhs_hamiltonian(M, a, z):
    z = np.ascontiguousarray(z, dtype=np.float64)
    f = np.zeros(8)
    lib().orc_rhs_hamiltonian(M, a, _p(z), _p(f))
    return f


def rhs_adm(M, a, z):
    z = np.ascontiguousarray(z, dtype=np.float64)
    f = np.zeros(8)
    lib().orc_rhs_adm(M, a, _p(z), _p(f))
    return f


def hamiltonian_adm(M, a, z):
    z = np.ascontiguousarray(z, dtype=np.float64)
    return lib().orc_hamiltonian_adm(M, a, _p(z))


def rk4_step_adm(M, a, h, z):
    z = np.array(z, dtype=np.float64)
    lib().orc_rk4_step_adm(M, a, h, _p(z))
    return z


def dopri5_tableau():
    c, a, b, bh = np.zeros(7), np.zeros(49), np.zeros(7), np.zeros(7)
    lib().orc_dopri5_tableau(_p(c), _p(a), _p(b), _p(bh))
    return c, a.reshape(7, 7), b, bh


def dopri5_linear(lam, h, y0):
    y5, e = _D(), _D()
    lib().orc_dopri5_linear_test(lam, h, y0, ctypes.byref(y5), ctypes.byref(e))
    return y5.value, e.value


def rk4_linear(lam, h, nsteps, y0):
    y = np.array([y0], dtype=np.float64)
    lib().orc_rk4_linear_test(lam, h, nsteps, _p(y))
    return y[0]


def rk4_step(M, a, h, y):
    y = np.array(y, dtype=np.float64)
    lib().orc_rk4_step(M, a, h, _p(y))
    return y


def rk4_step_hamiltonian(M, a, h, z):
    z = np.array(z, dtype=np.float64)
    lib().orc_rk4_step_hamiltonian(M, a, h, _p(z))
    return z


def trace_one(M, a, y0, term: Term, stride: int = 0):
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    y = np.zeros(8)
    lam = _D()
    st = _U32()
    traj = None
    if stride:
        ns = term.n_steps_cap // stride + 1
        traj = np.zeros((ns, 8))
    fate = lib().orc_trace_one(M, a, _p(y0), ctypes.byref(term), _p(y), ctypes.byref(lam),
                               ctypes.byref(st), _p(traj) if traj is not None else None,
                               stride)
    return {"y": y, "lambda": lam.value, "steps": st.value, "fate": fate, "traj": traj}


def trace_many(M, a, ics, term: Term, a_per_ray=None, stride: int = 0, nthreads: int = 0,
               want_traj: bool = False):
    """ics: (8, n) float64 SoA.  Returns a dict of numpy arrays."""
    ics = np.ascontiguousarray(ics, dtype=np.float64)
    n = ics.shape[1]
    y = np.zeros((8, n))
    lam = np.zeros(n)
    inv0 = np.zeros((4, n))
    inv1 = np.zeros((4, n))
    steps = np.zeros(n, dtype=np.uint32)
    fate = np.zeros(n, dtype=np.uint8)
    traj = None
    if want_traj and stride:
        traj = np.zeros((n, term.n_steps_cap // stride + 1, 8))
    apr = None if a_per_ray is None else np.ascontiguousarray(a_per_ray, dtype=np.float64)
    used = lib().orc_trace_many(M, a, _vp(apr), _p(ics), n, ctypes.byref(term), _p(y), _vp(lam),
                                _vp(inv0), _vp(inv1), _vp(steps), _vp(fate), _vp(traj),
                                stride if traj is not None else 0, nthreads)
    return {"y": y, "lambda": lam, "inv0": inv0, "inv1": inv1, "steps": steps, "fate": fate,
            "traj": traj, "threads": used}


def invariants(M, a, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    inv = np.zeros(4)
    lib().orc_invariants(M, a, _p(y), _p(inv))
    return inv


# ---------------------------------------------------------------- initial data
def paper_to_state(M, a, xp):
    xp = np.ascontiguousarray(xp, dtype=np.float64)
    y = np.zeros(8)
    lib().orc_paper_to_state(M, a, _p(xp), _p(y))
    return y


def state_to_momenta(M, a, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    p = np.zeros(4)
    lib().orc_state_to_momenta(M, a, _p(y), _p(p))
    return p


def bl_to_cartesian(a, r, th, ph):
    xyz = np.zeros(3)
    lib().orc_bl_to_cartesian(a, r, th, ph, _p(xyz))
    return xyz


def schw_circular(M, r):
    E, L = _D(), _D()
    lib().orc_schw_circular(M, r, ctypes.byref(E), ctypes.byref(L))
    return E.value, L.value


def schw_gralorbits(k, M=1.0):
    pt, pp = _D(), _D()
    lib().orc_schw_gralorbits(k, M, ctypes.byref(pt), ctypes.byref(pp))
    return pt.value, pp.value


def kerr_circular_paper(M, a, r, sgn):
    E, L = _D(), _D()
    lib().orc_kerr_circular_paper(M, a, r, int(sgn), ctypes.byref(E), ctypes.byref(L))
    return E.value, L.value


def kerr_circular_bardeen(M, a, r, prograde):
    E, L = _D(), _D()
    lib().orc_kerr_circular_bardeen(M, a, r, int(prograde), ctypes.byref(E), ctypes.byref(L))
    return E.value, L.value


def kerr_omega(M, a, r, pt_paper, pphi):
    return lib().orc_kerr_omega(M, a, r, pt_paper, pphi)


def isco_bardeen(M, a, prograde):
    return lib().orc_isco_bardeen(M, a, int(prograde))


def isco_paper_literal(M, a, sgn):
    return lib().orc_isco_paper_literal(M, a, int(sgn))


def dEdr_root(M, a, prograde, r_lo, r_hi):
    return lib().orc_dEdr_numeric_root(M, a, int(prograde), r_lo, r_hi)


def photon_orbit(M, a, prograde):
    return lib().orc_photon_orbit(M, a, int(prograde))


def circular_state(M, a, r, prograde):
    y = np.zeros(8)
    lib().orc_circular_state(M, a, r, int(prograde), _p(y))
    return y


def camera_ic(M, a, r_o, th_o, fov_half, nx, ny, pix):
    y = np.zeros(8)
    lib().orc_camera_ic(M, a, r_o, th_o, fov_half, nx, ny, int(pix), _p(y))
    return y


def camera_ics(M, a, r_o, th_o, fov_half, nx, ny, pixels):
    pixels = np.asarray(pixels, dtype=np.uint64)
    out = np.zeros((8, len(pixels)))
    for k, pix in enumerate(pixels):
        out[:, k] = camera_ic(M, a, r_o, th_o, fov_half, nx, ny, int(pix))
    return out


def critical_curve_distance(M, a, th_o, alpha, beta):
    return lib().orc_critical_curve_distance(M, a, th_o, alpha, beta)


def critical_curve_polyline(M, a, th_o, n=200_000):
    """The Kerr critical curve as a closed polyline of 2n (alpha, beta) points
    (orc_critical_curve_polyline)."""
    al = np.empty(2 * n)
    be = np.empty(2 * n)
    lib().orc_critical_curve_polyline(M, a, th_o, int(n), _p(al), _p(be))
    return al, be


def critical_curve_distance_many(M, a, th_o, alpha, beta, n=20_000, upper=0.25):
    """Distance of many (alpha, beta) points to the critical curve at once:
    the nearest vertex of the dense polyline (k-d tree), then the exact
    distance to the two polyline segments at that vertex.  Agrees with
    critical_curve_distance to well below the polyline spacing.  Points
    farther than `upper` from every vertex get +inf (a nearest-neighbour
    search from far away is slow, and callers only compare with a small
    exclusion distance)."""
    from scipy.spatial import cKDTree

    cal, cbe = critical_curve_polyline(M, a, th_o, n)
    pts = np.stack([cal, cbe], axis=1)
    q = np.stack([np.asarray(alpha, dtype=np.float64).ravel(), np.asarray(beta, dtype=np.float64).ravel()], axis=1)
    d, k = cKDTree(pts).query(q, distance_upper_bound=upper)
    far = ~np.isfinite(d)
    k = np.where(far, 0, k)
    m = len(pts)
    best = d
    for nb in ((k - 1) % m, (k + 1) % m):
        p0, p1 = pts[k], pts[nb]
        seg = p1 - p0
        L2 = np.einsum("ij,ij->i", seg, seg)
        t = np.where(L2 > 0, np.einsum("ij,ij->i", q - p0, seg) / np.where(L2 > 0, L2, 1.0), 0.0)
        t = np.clip(t, 0.0, 1.0)
        proj = p0 + t[:, None] * seg
        best = np.minimum(best, np.hypot(q[:, 0] - proj[:, 0], q[:, 1] - proj[:, 1]))
    best[far] = np.inf
    return best.reshape(np.shape(alpha))


def splitmix64(seed, counter):
    return lib().orc_splitmix64(seed, counter)


def uniform(seed, counter):
    return lib().orc_uniform(seed, counter)


def radial_potential(M, a, E, Lz, Q, r):
    return lib().orc_radial_potential(M, a, E, Lz, Q, r)


def bound_orbit_solve(M, a, rp, e, iota):
    E, Lz, Q, r3 = _D(), _D(), _D(), _D()
    code = lib().orc_bound_orbit_solve(M, a, rp, e, iota, ctypes.byref(E), ctypes.byref(Lz),
                                       ctypes.byref(Q), ctypes.byref(r3))
    return code, E.value, Lz.value, Q.value, r3.value


def bound_sample(M, a_max, seed, index, spin_fixed=False):
    a = _D()
    y = np.zeros(8)
    cand = np.zeros(4)
    j = lib().orc_bound_sample(M, a_max, int(spin_fixed), seed, int(index), ctypes.byref(a), _p(y),
                               _p(cand))
    return {"a": a.value, "y": y, "accepted": j, "cand": cand}


def bound_samples(M, a_max, seed, indices, spin_fixed=False):
    indices = np.asarray(indices)
    n = len(indices)
    ys = np.zeros((8, n))
    spins = np.zeros(n)
    acc = np.zeros(n, dtype=np.int64)
    for k, i in enumerate(indices):
        s = bound_sample(M, a_max, seed, int(i), spin_fixed)
        ys[:, k] = s["y"]
        spins[k] = s["a"]
        acc[k] = s["accepted"]
    return ys, spins, acc

"""Python binding of libmalbec.so: argument marshalling only.

Every step of the geodesic path runs in the library's CUDA kernels; this module
allocates device buffers with PyTorch, passes raw pointers and the current CUDA
stream through ctypes, and returns tensor views into the library's output
layout.  There is no CPU fallback: if the library is missing or no GPU is
present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmalbec.so")

FP64, FP32_MIXED = 0, 1
FORM_GEODESIC, FORM_HAMILTONIAN, FORM_ADM = 0, 1, 2
METHOD_RK4, METHOD_DOPRI5 = 0, 1
OUT_FINAL, OUT_STRIDED, OUT_STRIDED_CARTESIAN = 0, 1, 2
FATE_CAPTURED, FATE_ESCAPED, FATE_CAPPED, FATE_NONFINITE = 1, 2, 3, 4
FATE_DRIFTED, FATE_MASK, NORM_DRIFT_TOL = 0x80, 0x7F, 1e-3  # validity flag or-ed into a fate
OK, EINVAL, ENOMEM, EBUSY, ETIMEDOUT, ECUDA, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6

_D = ctypes.c_double
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t
_VP = ctypes.c_void_p


class Metric(ctypes.Structure):
    _fields_ = [("M", _D), ("a", _D), ("a_per_ray", _VP)]


class Term(ctypes.Structure):
    _fields_ = [("eps_hor", _D), ("r_esc", _D), ("n_steps_cap", _U32), ("dl", _D), ("dl_r_scale", _D),
                ("form", _U32), ("method", _U32), ("rtol", _D), ("atol", _D)]


class Camera(ctypes.Structure):
    _fields_ = [("r_obs", _D), ("incl", _D), ("fov_half", _D), ("nx", _U32), ("ny", _U32)]


class Layout(ctypes.Structure):
    _fields_ = [("y", _SZ), ("lam", _SZ), ("inv0", _SZ), ("inv1", _SZ), ("steps", _SZ), ("fate", _SZ),
                ("traj", _SZ), ("n_samples", _U64), ("total", _SZ)]


class CameraLayout(ctypes.Structure):
    _fields_ = [("fate", _SZ), ("steps", _SZ), ("theta", _SZ), ("phi", _SZ), ("total", _SZ)]


class MixedZone(ctypes.Structure):
    _fields_ = [("horizon_factor", _D), ("photon_margin", _D), ("pole_sin", _D)]


BUNDLE_STATES, BUNDLE_CAMERA, BUNDLE_BOUND = 0, 1, 2


class Bundle(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n", _U32), ("M", _D), ("a", _D), ("term", Term), ("camera", Camera),
                ("ics", _VP), ("seed", _U64), ("out", _VP)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("threads_per_block", _U32), ("blocks_per_sm", _U32), ("refill_min", _U32),
                ("zone_batch", _U32), ("zone_wait", _U32), ("exchange", _U32), ("zone_wait_limit_us", _U32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", _SZ), ("max_active", _U32), ("max_pending", _U32), ("precision", ctypes.c_int),
                ("idle_timeout_s", _D), ("form", _U32), ("method", _U32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _U64), ("admitted", _U64), ("completed", _U64), ("released", _U64),
                ("pending", _U64), ("active", _U64), ("bytes_in_use", _U64), ("kernel_launches", _U64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class MalbecError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = f"{where}: {strerror(code)}"
        if code == ECUDA:
            msg += f" ({last_cuda_error()})"
        super().__init__(msg)


_lib = None


def lib() -> ctypes.CDLL:
    """Load libmalbec.so (built by paper_1803_08320_gb300.build).  Raises if it
    has not been built: there is no fallback path."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found: build it with `python -m paper_1803_08320_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    def sig(name, res, *args):
        f = getattr(L, name)
        f.restype = res
        f.argtypes = list(args)

    sig("malbec_strerror", ctypes.c_char_p, ctypes.c_int)
    sig("malbec_last_cuda_error", ctypes.c_char_p)
    sig("malbec_build_info", ctypes.c_char_p)
    sig("malbec_out_layout", ctypes.c_int, ctypes.c_int, ctypes.c_int, _U64, _U32, _U32, ctypes.POINTER(Layout))
    sig("malbec_out_bytes", _SZ, ctypes.c_int, ctypes.c_int, _U64, _U32, _U32)
    sig("malbec_trace", ctypes.c_int, Metric, _VP, _U64, Term, ctypes.c_int, _U32, ctypes.c_int, _VP, _VP)
    sig("malbec_trace_noalloc", ctypes.c_int, Metric, _VP, _U64, Term, ctypes.c_int, _U32, ctypes.c_int, _VP, _VP)
    sig("malbec_camera_out_layout", ctypes.c_int, ctypes.POINTER(Camera), ctypes.POINTER(CameraLayout))
    sig("malbec_trace_camera", ctypes.c_int, Metric, ctypes.POINTER(Camera), Term, ctypes.c_int, _VP, _VP)
    sig("malbec_ic_camera", ctypes.c_int, Metric, ctypes.POINTER(Camera), _VP, _U64, _VP, _VP)
    sig("malbec_ic_circular", ctypes.c_int, Metric, _VP, _U64, ctypes.c_int, _VP, _VP)
    sig("malbec_ic_from_paper", ctypes.c_int, Metric, _VP, _U64, _VP, _VP)
    sig("malbec_ic_bound", ctypes.c_int, _D, _D, ctypes.c_int, _U64, _U64, _U64, _VP, _VP, _VP, _VP)
    sig("malbec_invariants", ctypes.c_int, Metric, _VP, _U64, _VP, _VP)
    sig("malbec_measure_fma_peak", ctypes.c_int, ctypes.c_int, ctypes.POINTER(_D))
    sig("malbec_measure_step_loop", ctypes.c_int, _U32, ctypes.POINTER(_D))
    sig("malbec_check_fp64_helpers", ctypes.c_int, ctypes.POINTER(_D))
    sig("malbec_check_operand_forms", ctypes.c_int, ctypes.POINTER(_U64))
    sig("malbec_bundle_out_bytes", _SZ, ctypes.POINTER(Bundle), ctypes.c_int)
    sig("malbec_trace_bundles", ctypes.c_int, ctypes.POINTER(Bundle), _U32, ctypes.c_int, _VP)
    sig("malbec_plan_create", ctypes.c_int, ctypes.POINTER(Bundle), _U32, ctypes.c_int, ctypes.POINTER(_VP))
    sig("malbec_plan_launch", ctypes.c_int, _VP, _VP)
    sig("malbec_plan_autotune", ctypes.c_int, _VP, _VP, ctypes.POINTER(LaunchConfig))
    sig("malbec_plan_destroy", ctypes.c_int, _VP)
    sig("malbec_server_create", ctypes.c_int, ctypes.POINTER(ServerConfig), ctypes.POINTER(_VP))
    sig("malbec_server_destroy", ctypes.c_int, _VP)
    sig("malbec_submit", ctypes.c_int, _VP, ctypes.POINTER(Bundle), ctypes.POINTER(_U64))
    sig("malbec_poll", ctypes.c_int, _VP, _U64, ctypes.POINTER(ctypes.c_int))
    sig("malbec_job_output", ctypes.c_int, _VP, _U64, ctypes.POINTER(_VP), ctypes.POINTER(_SZ))
    sig("malbec_job_copy_output", ctypes.c_int, _VP, _U64, _VP, _SZ, _VP)
    sig("malbec_job_release", ctypes.c_int, _VP, _U64)
    sig("malbec_server_stats_get", ctypes.c_int, _VP, ctypes.POINTER(ServerStats))
    sig("malbec_set_launch_config", ctypes.c_int, ctypes.POINTER(LaunchConfig))
    sig("malbec_get_launch_config", ctypes.c_int, ctypes.POINTER(LaunchConfig))
    sig("malbec_set_mixed_zone", ctypes.c_int, ctypes.POINTER(MixedZone))
    sig("malbec_wait_status", ctypes.c_int, ctypes.POINTER(_U64))
    sig("malbec_get_mixed_zone", ctypes.c_int, ctypes.POINTER(MixedZone))


def strerror(code: int) -> str:
    return lib().malbec_strerror(code).decode()


def last_cuda_error() -> str:
    return lib().malbec_last_cuda_error().decode()


def build_info() -> str:
    return lib().malbec_build_info().decode()


def _check(code: int, where: str):
    if code != OK:
        raise MalbecError(code, where)


def _torch():
    import torch

    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return _VP(s.cuda_stream)


def _ptr(t):
    return None if t is None else _VP(t.data_ptr())


def _dev_f64(x, n_expected=None):
    torch = _torch()
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(np.asarray(x, dtype=np.float64))
    if x.device.type != "cuda":
        x = x.to("cuda")
    x = x.to(torch.float64).contiguous()
    return x


@dataclass
class Termination:
    eps_hor: float = 0.01
    r_esc: float = 1100.0
    n_steps_cap: int = 10_000
    dl: float = 0.01
    dl_r_scale: float = 0.0
    form: int = 0  # FORM_GEODESIC, FORM_HAMILTONIAN or FORM_ADM
    method: int = 0  # METHOD_RK4 or METHOD_DOPRI5 (adaptive; rtol, atol)
    rtol: float = 0.0
    atol: float = 0.0

    def c(self) -> Term:
        return Term(float(self.eps_hor), float(self.r_esc), int(self.n_steps_cap), float(self.dl),
                    float(self.dl_r_scale), int(self.form), int(self.method), float(self.rtol), float(self.atol))


def term_from(t, form=None, method=None, rtol=None, atol=None) -> Termination:
    """A Termination from any object with the same fields (e.g. a workload's
    term), optionally with another form or integrator."""
    if isinstance(t, Termination) and form is None and method is None and rtol is None and atol is None:
        return t
    f = getattr(t, "form", 0) if form is None else form
    m = getattr(t, "method", 0) if method is None else method
    rt = getattr(t, "rtol", 0.0) if rtol is None else rtol
    at = getattr(t, "atol", 0.0) if atol is None else atol
    return Termination(t.eps_hor, t.r_esc, t.n_steps_cap, t.dl, t.dl_r_scale, int(f), int(m), float(rt), float(at))


def _prec(p) -> int:
    if isinstance(p, str):
        return {"fp64": FP64, "fp32_mixed": FP32_MIXED, "mixed": FP32_MIXED}[p]
    return int(p)


def out_layout(mode: int, precision, n: int, n_steps_cap: int, stride: int) -> Layout:
    L = Layout()
    _check(lib().malbec_out_layout(mode, _prec(precision), n, n_steps_cap, stride, ctypes.byref(L)),
           "malbec_out_layout")
    return L


def _views_final(buf, L: Layout, n: int, mode: int, precision):
    torch = _torch()

    def v(off, count, dtype, shape):
        itemsize = torch.empty((), dtype=dtype).element_size()
        return buf[off: off + count * itemsize].view(dtype).view(*shape)

    out = {
        "y": v(L.y, 8 * n, torch.float64, (8, n)),
        "lambda": v(L.lam, n, torch.float64, (n,)),
        "inv0": v(L.inv0, 4 * n, torch.float64, (4, n)),
        "inv1": v(L.inv1, 4 * n, torch.float64, (4, n)),
        "steps": v(L.steps, n, torch.int32, (n,)),
        "fate": v(L.fate, n, torch.uint8, (n,)),
        "buffer": buf,
    }
    if mode != OUT_FINAL:
        ns = int(L.n_samples)
        comps = 4 if mode == OUT_STRIDED_CARTESIAN else 8
        dt = torch.float64 if _prec(precision) == FP64 else torch.float32
        out["traj"] = v(L.traj, n * ns * comps, dt, (n, ns, comps))
    return out


def check_device_tensor(t, name: str, dtype, numel_min: int = None, numel: int = None, shape=None,
                        device_type: str = "cuda", device_index=None):
    """Raise ValueError unless `t` is a contiguous tensor of `dtype` on the
    given device with the given shape or element count.  The library sees raw
    pointers only and cannot check sizes: a short or misplaced buffer would
    make a kernel read or write out of bounds, so the binding checks before
    any call."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if t.device.type != device_type:
        raise ValueError(f"{name}: expected a {device_type} tensor, got one on {t.device}")
    if device_index is not None and t.device.index != device_index:
        raise ValueError(f"{name}: on {t.device}, but the current device is {device_type}:{device_index}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    if numel_min is not None and t.numel() < numel_min:
        raise ValueError(f"{name}: needs at least {numel_min} elements, got {t.numel()}")


def _current_device_index():
    torch = _torch()
    return torch.cuda.current_device() if torch.cuda.is_available() else None


def trace(M: float, a: float, ics, term, mode: int = OUT_FINAL, stride: int = 0, precision="fp64",
          a_per_ray=None, stream=None, out=None):
    """Integrate the rays `ics` ((8, n) float64 on the GPU, SoA).  Returns a
    dict of views: y (8, n), lambda, inv0 (4, n), inv1 (4, n), steps (int32
    view of the uint32 field), fate, [traj (n, n_samples, 8)].  `out`, if
    given, is a contiguous uint8 CUDA tensor of at least out_layout(...).total
    bytes on the same device as `ics`."""
    torch = _torch()
    ics = _dev_f64(ics)
    n = ics.shape[1]
    t = term_from(term)
    L = out_layout(mode, precision, n, t.n_steps_cap, stride if mode != OUT_FINAL else 0)
    if out is None:
        out = torch.empty(L.total, dtype=torch.uint8, device=ics.device)
    else:
        check_device_tensor(out, "out", torch.uint8, numel_min=int(L.total), device_index=ics.device.index)
    apr = None if a_per_ray is None else _dev_f64(a_per_ray)
    if apr is not None:
        check_device_tensor(apr, "a_per_ray", torch.float64, numel=n, device_index=ics.device.index)
    m = Metric(float(M), float(a), _ptr(apr))
    _check(lib().malbec_trace(m, _ptr(ics), n, t.c(), mode, stride if mode != OUT_FINAL else 0,
                              _prec(precision), _ptr(out), _stream(stream)), "malbec_trace")
    res = _views_final(out, L, n, mode, precision)
    res["_keep"] = (ics, apr)
    return res


def trace_noalloc(M: float, a: float, ics, term, out, mode: int = OUT_FINAL, stride: int = 0,
                  precision="fp64", a_per_ray=None, stream=None):
    """`trace` through malbec_trace_noalloc, for callers that cannot allocate
    device memory: `out` (a contiguous uint8 CUDA tensor of at least
    out_layout(...).total bytes), `ics` (contiguous float64, shape (8, n)) and
    `a_per_ray` (contiguous float64, n elements, or None) must already be on
    the current device; they are checked here, without copies, and a bad one
    raises ValueError before anything runs.  The library uses its static
    work-queue block and allocates nothing.  Calls that overlap on the GPU
    share that block and race: serialise them."""
    torch = _torch()
    dev = _current_device_index()
    check_device_tensor(ics, "ics", torch.float64, device_index=dev)
    if ics.dim() != 2 or ics.shape[0] != 8 or ics.shape[1] < 1:
        raise ValueError(f"ics: expected shape (8, n) with n >= 1, got {tuple(ics.shape)}")
    t = term_from(term)
    n = ics.shape[1]
    L = out_layout(mode, precision, n, t.n_steps_cap, stride if mode != OUT_FINAL else 0)
    check_device_tensor(out, "out", torch.uint8, numel_min=int(L.total), device_index=dev)
    if a_per_ray is not None:
        check_device_tensor(a_per_ray, "a_per_ray", torch.float64, numel=n, device_index=dev)
    m = Metric(float(M), float(a), _ptr(a_per_ray))
    _check(lib().malbec_trace_noalloc(m, _ptr(ics), n, t.c(), mode, stride if mode != OUT_FINAL else 0,
                                      _prec(precision), _ptr(out), _stream(stream)), "malbec_trace_noalloc")
    return _views_final(out, L, n, mode, precision)


def make_bundle(kind: int, n: int, M: float, a: float, term, camera: Camera | None = None, ics=None,
                seed: int = 0) -> Bundle:
    """Describe one bundle (outputs attached by `attach_outputs`)."""
    b = Bundle()
    b.kind = int(kind)
    b.n = int(n)
    b.M = float(M)
    b.a = float(a)
    b.term = term_from(term).c()
    if camera is not None:
        b.camera = camera
    b.ics = None if ics is None else _VP(ics.data_ptr())
    b.seed = int(seed) & (2**64 - 1)
    return b


def bundle_views(b: Bundle, buf, precision):
    """Tensor views into a bundle's output buffer."""
    torch = _torch()
    n = int(b.n)
    if b.kind == BUNDLE_CAMERA:
        L = camera_layout(Camera(1000.0, 1.0, 1.0, n, 1))
        return {"fate": buf[L.fate: L.fate + n], "steps": buf[L.steps: L.steps + 4 * n].view(torch.int32),
                "theta": buf[L.theta: L.theta + 8 * n].view(torch.float64),
                "phi": buf[L.phi: L.phi + 8 * n].view(torch.float64), "buffer": buf}
    L = out_layout(OUT_FINAL, precision, n, int(b.term.n_steps_cap), 0)
    return _views_final(buf, L, n, OUT_FINAL, precision)


def attach_outputs(bundles, precision):
    """Allocate (torch) and attach an output buffer to every bundle; returns
    the per-bundle views."""
    torch = _torch()
    views = []
    for b in bundles:
        nbytes = lib().malbec_bundle_out_bytes(ctypes.byref(b), _prec(precision))
        if nbytes == 0:
            raise MalbecError(EINVAL, "malbec_bundle_out_bytes")
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        b.out = _VP(buf.data_ptr())
        views.append(bundle_views(b, buf, precision))
    return views


def _bundle_array(bundles):
    arr = (Bundle * len(bundles))()
    for i, b in enumerate(bundles):
        arr[i] = b
    return arr


def trace_bundles(bundles, precision="fp64", stream=None):
    """Trace a list of Bundle (outputs attached) in one persistent launch."""
    arr = _bundle_array(bundles)
    _check(lib().malbec_trace_bundles(arr, len(bundles), _prec(precision), _stream(stream)), "malbec_trace_bundles")


class Plan:
    """Bundles uploaded once; launch replayed as a CUDA graph."""

    def __init__(self, bundles, precision="fp64"):
        self._arr = _bundle_array(bundles)
        self._h = _VP()
        _check(lib().malbec_plan_create(self._arr, len(bundles), _prec(precision), ctypes.byref(self._h)),
               "malbec_plan_create")

    def launch(self, stream=None):
        _check(lib().malbec_plan_launch(self._h, _stream(stream)), "malbec_plan_launch")

    def autotune(self, stream=None) -> dict:
        best = LaunchConfig()
        _check(lib().malbec_plan_autotune(self._h, _stream(stream), ctypes.byref(best)), "malbec_plan_autotune")
        return best.as_dict()

    def close(self):
        if self._h:
            lib().malbec_plan_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (malbec_server_*)."""

    def __init__(self, hbm_budget: int = 150 * 10**9, max_active: int = 1024, max_pending: int = 100_000,
                 precision="fp32_mixed", idle_timeout_s: float = 0.002, form: int = FORM_GEODESIC,
                 method: int = METHOD_RK4):
        """form, method: the class of every job of this server (a job's
        term.form and term.method must match)."""
        self.precision = precision
        cfg = ServerConfig(int(hbm_budget), int(max_active), int(max_pending), _prec(precision),
                           float(idle_timeout_s), int(form), int(method))
        self._h = _VP()
        _check(lib().malbec_server_create(ctypes.byref(cfg), ctypes.byref(self._h)), "malbec_server_create")
        self._specs = {}

    def submit(self, bundle: Bundle) -> int:
        jid = _U64()
        _check(lib().malbec_submit(self._h, ctypes.byref(bundle), ctypes.byref(jid)), "malbec_submit")
        self._specs[jid.value] = bundle
        return jid.value

    def try_submit(self, bundle: Bundle):
        """submit, or None when the admission queue is full."""
        jid = _U64()
        rc = lib().malbec_submit(self._h, ctypes.byref(bundle), ctypes.byref(jid))
        if rc == EBUSY:
            return None
        _check(rc, "malbec_submit")
        self._specs[jid.value] = bundle
        return jid.value

    def poll(self, job_id: int) -> bool:
        d = ctypes.c_int()
        _check(lib().malbec_poll(self._h, job_id, ctypes.byref(d)), "malbec_poll")
        return bool(d.value)

    def output(self, job_id: int, stream=None):
        """Copy a finished job's output into a new CUDA tensor; returns views."""
        torch = _torch()
        ptr, nbytes = _VP(), _SZ()
        _check(lib().malbec_job_output(self._h, job_id, ctypes.byref(ptr), ctypes.byref(nbytes)), "malbec_job_output")
        buf = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        _check(lib().malbec_job_copy_output(self._h, job_id, _VP(buf.data_ptr()), nbytes.value, _stream(stream)),
               "malbec_job_copy_output")
        return bundle_views(self._specs[job_id], buf, self.precision)

    def release(self, job_id: int):
        # copies of the output made with `output` run on the current stream
        _torch().cuda.current_stream().synchronize()
        _check(lib().malbec_job_release(self._h, job_id), "malbec_job_release")
        self._specs.pop(job_id, None)

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().malbec_server_stats_get(self._h, ctypes.byref(s)), "malbec_server_stats_get")
        return s.as_dict()

    def close(self):
        if self._h:
            lib().malbec_server_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def camera_layout(cam: Camera) -> CameraLayout:
    L = CameraLayout()
    _check(lib().malbec_camera_out_layout(ctypes.byref(cam), ctypes.byref(L)), "malbec_camera_out_layout")
    return L


def make_camera(r_obs, incl, fov_half, nx, ny) -> Camera:
    return Camera(float(r_obs), float(incl), float(fov_half), int(nx), int(ny))


def trace_camera(M: float, a: float, cam: Camera, term, precision="fp64", stream=None, out=None):
    """Render the backward camera.  Returns views fate (n,), steps, theta, phi."""
    torch = _torch()
    L = camera_layout(cam)
    n = cam.nx * cam.ny
    if out is None:
        out = torch.empty(L.total, dtype=torch.uint8, device="cuda")
    _check(lib().malbec_trace_camera(Metric(float(M), float(a), None), ctypes.byref(cam), term_from(term).c(),
                                     _prec(precision), _ptr(out), _stream(stream)), "malbec_trace_camera")
    return {
        "fate": out[L.fate: L.fate + n],
        "steps": out[L.steps: L.steps + 4 * n].view(torch.int32),
        "theta": out[L.theta: L.theta + 8 * n].view(torch.float64),
        "phi": out[L.phi: L.phi + 8 * n].view(torch.float64),
        "buffer": out,
    }


def ic_camera(M: float, a: float, cam: Camera, pixels, stream=None):
    torch = _torch()
    px = torch.as_tensor(np.asarray(pixels, dtype=np.int64)).to("cuda")
    n = px.numel()
    ics = torch.empty((8, n), dtype=torch.float64, device="cuda")
    _check(lib().malbec_ic_camera(Metric(float(M), float(a), None), ctypes.byref(cam), _ptr(px), n, _ptr(ics),
                                  _stream(stream)), "malbec_ic_camera")
    return ics


def read_paper_rows(path: str) -> np.ndarray:
    """Initial-condition rows in the paper's text layout (Sec. 5: one ray per
    line, t r theta phi p_t p_r p_theta p_phi, the p_t column holding E > 0;
    blank lines and '#' comments skipped): a (8, n) float64 array."""
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            vals = [float(v) for v in line.split()]
            if len(vals) != 8:
                raise ValueError(f"{path}: expected 8 columns, got {len(vals)}: {line!r}")
            rows.append(vals)
    if not rows:
        raise ValueError(f"{path}: no rows")
    return np.ascontiguousarray(np.array(rows, dtype=np.float64).T)


def ic_from_paper(M: float, a: float, rows, a_per_ray=None, stream=None):
    """States (x, u) on the device from the paper's rows ((8, n), p_t column =
    E): malbec_ic_from_paper."""
    torch = _torch()
    r = _dev_f64(rows)
    n = r.shape[1]
    ics = torch.empty((8, n), dtype=torch.float64, device="cuda")
    apr = None if a_per_ray is None else _dev_f64(a_per_ray)
    _check(lib().malbec_ic_from_paper(Metric(float(M), float(a), _ptr(apr)), _ptr(r), n, _ptr(ics),
                                      _stream(stream)), "malbec_ic_from_paper")
    return ics


def ic_circular(M: float, a: float, radii, prograde: bool = True, stream=None):
    torch = _torch()
    r = _dev_f64(radii)
    n = r.numel()
    ics = torch.empty((8, n), dtype=torch.float64, device="cuda")
    _check(lib().malbec_ic_circular(Metric(float(M), float(a), None), _ptr(r), n, int(bool(prograde)), _ptr(ics),
                                    _stream(stream)), "malbec_ic_circular")
    return ics


def ic_bound(M: float, a_max: float, seed: int, n: int, index0: int = 0, spin_fixed: bool = False, stream=None):
    """Generic bound-orbit ensemble: returns (ics (8, n), spins (n,), accepted (n,) int32)."""
    torch = _torch()
    ics = torch.empty((8, n), dtype=torch.float64, device="cuda")
    spins = torch.empty(n, dtype=torch.float64, device="cuda")
    acc = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(lib().malbec_ic_bound(float(M), float(a_max), int(bool(spin_fixed)), int(seed) & (2**64 - 1),
                                 int(index0), int(n), _ptr(ics), _ptr(spins), _ptr(acc), _stream(stream)),
           "malbec_ic_bound")
    return ics, spins, acc


def invariants(M: float, a: float, states, a_per_ray=None, stream=None):
    torch = _torch()
    y = _dev_f64(states)
    n = y.shape[1]
    inv = torch.empty((4, n), dtype=torch.float64, device="cuda")
    apr = None if a_per_ray is None else _dev_f64(a_per_ray)
    _check(lib().malbec_invariants(Metric(float(M), float(a), _ptr(apr)), _ptr(y), n, _ptr(inv), _stream(stream)),
           "malbec_invariants")
    return inv


def set_mixed_zone(horizon_factor=None, photon_margin=None, pole_sin=None, reset=False):
    """Change the FP64 zone of the FP32_MIXED path (None keeps a field)."""
    if reset:
        _check(lib().malbec_set_mixed_zone(None), "malbec_set_mixed_zone")
        return get_mixed_zone()
    z = get_mixed_zone()
    if horizon_factor is not None:
        z.horizon_factor = float(horizon_factor)
    if photon_margin is not None:
        z.photon_margin = float(photon_margin)
    if pole_sin is not None:
        z.pole_sin = float(pole_sin)
    _check(lib().malbec_set_mixed_zone(ctypes.byref(z)), "malbec_set_mixed_zone")
    return z


def set_launch_config(threads_per_block=0, blocks_per_sm=0, refill_min=0, zone_batch=0, zone_wait=0, exchange=0,
                      zone_wait_limit_us=0, reset=False) -> LaunchConfig:
    """Process-wide launch configuration of the trace kernels (0 = automatic)."""
    if reset:
        _check(lib().malbec_set_launch_config(None), "malbec_set_launch_config")
    else:
        c = LaunchConfig(int(threads_per_block), int(blocks_per_sm), int(refill_min), int(zone_batch),
                         int(zone_wait), int(exchange), int(zone_wait_limit_us))
        _check(lib().malbec_set_launch_config(ctypes.byref(c)), "malbec_set_launch_config")
    return get_launch_config()


def wait_status():
    """(timed_out, total): malbec_wait_status -- whether a bounded device
    wait ran out since the previous call (MALBEC_ETIMEDOUT), and the device's
    running count of such expiries.  Synchronises the device."""
    t = _U64()
    rc = lib().malbec_wait_status(ctypes.byref(t))
    if rc not in (OK, ETIMEDOUT):
        _check(rc, "malbec_wait_status")
    return rc == ETIMEDOUT, int(t.value)


def get_launch_config() -> LaunchConfig:
    c = LaunchConfig()
    _check(lib().malbec_get_launch_config(ctypes.byref(c)), "malbec_get_launch_config")
    return c


def get_mixed_zone() -> MixedZone:
    z = MixedZone()
    _check(lib().malbec_get_mixed_zone(ctypes.byref(z)), "malbec_get_mixed_zone")
    return z


def measure_fma_peak(precision="fp64") -> float:
    """Measured FMA GFLOP/s of the current GPU (blocks the caller)."""
    g = _D()
    _check(lib().malbec_measure_fma_peak(_prec(precision), ctypes.byref(g)), "malbec_measure_fma_peak")
    return g.value


def measure_step_loop(form=FORM_GEODESIC) -> float:
    """RK4 steps/s of the bare FP64 step loop of one form (blocks the caller):
    the ceiling of the trace kernels for that right-hand side."""
    g = _D()
    _check(lib().malbec_measure_step_loop(int(form), ctypes.byref(g)), "malbec_measure_step_loop")
    return g.value


def check_fp64_helpers() -> dict:
    """Max errors of the FP64 stage sine/cosine, reciprocal and step
    sine/cosine against CUDA's sincos and IEEE division (blocks the caller)."""
    e = (_D * 6)()
    _check(lib().malbec_check_fp64_helpers(e), "malbec_check_fp64_helpers")
    return {"sin_abs": e[0], "cos_abs": e[1], "recip_ulp": e[2], "recip_estimate_rel": e[3],
            "step_sin_abs": e[4], "step_cos_abs": e[5]}


def check_operand_forms() -> dict:
    """Mismatch counts of the kernels' operand forms against the plain
    operations, bit for bit (blocks the caller): FP64 fma(x, y, -0),
    fma(x, 1, y), fma(x, 1, -y), the exponent doubling, and the paired FP32
    add, subtract, multiply/fma and compensated update."""
    c = (_U64 * 8)()
    _check(lib().malbec_check_operand_forms(c), "malbec_check_operand_forms")
    keys = ("fp64_mul", "fp64_add", "fp64_sub", "fp64_twice", "fp32x2_add", "fp32x2_sub", "fp32x2_mul_fma",
            "fp32x2_comp_add")
    return dict(zip(keys, (int(v) for v in c)))

// api.cu -- extern "C" entry points of libmalbec.so (see include/malbec.h):
// argument validation, output layouts, per-call scratch from the
// stream-ordered allocator, launch shapes, error reporting and the FMA
// peak measurement.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "internal.h"

namespace malbec {

namespace {
thread_local std::string g_last_cuda_error = "no error";

size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

bool finite_pos(double x) { return isfinite(x) && x > 0.0; }

double host_r_plus(double M, double a) { return M + sqrt(M * M - a * a); }

}  // namespace

int check_metric(const malbec_metric& m) {
  if (!finite_pos(m.M) || !isfinite(m.a) || m.a < 0.0 || !(m.a < m.M)) return MALBEC_EINVAL;
  return MALBEC_OK;
}

// The capture radius is largest for a = 0 (r_+ = 2M); with per-ray spins the
// escape radius must clear that worst case.
int check_term(const malbec_term& t, const malbec_metric& m) {
  if (!isfinite(t.eps_hor) || t.eps_hor < 0.0) return MALBEC_EINVAL;
  if (t.form != MALBEC_FORM_GEODESIC && t.form != MALBEC_FORM_HAMILTONIAN && t.form != MALBEC_FORM_ADM)
    return MALBEC_EINVAL;
  const bool scaled = t.dl_r_scale != 0.0;
  if (scaled && !finite_pos(t.dl_r_scale)) return MALBEC_EINVAL;
  if (!scaled && !finite_pos(t.dl)) return MALBEC_EINVAL;
  const double rp = m.a_per_ray ? 2.0 * m.M : host_r_plus(m.M, m.a);
  if (!isfinite(t.r_esc) || !(t.r_esc > (1.0 + t.eps_hor) * rp)) return MALBEC_EINVAL;
  if (t.method != MALBEC_METHOD_RK4 && t.method != MALBEC_METHOD_DOPRI5) return MALBEC_EINVAL;
  if (t.method == MALBEC_METHOD_DOPRI5) {
    if (!finite_pos(t.atol) || !isfinite(t.rtol) || t.rtol < 0.0) return MALBEC_EINVAL;
    if (scaled && (!isfinite(t.dl) || t.dl < 0.0)) return MALBEC_EINVAL;
  }
  return MALBEC_OK;
}

// The adaptive method runs in FP64 on every entry point, and in FP32_MIXED
// (its FP32 error estimate carries rounding noise of ~1e-7 of the state)
// when rtol >= MALBEC_DOPRI5_MIXED_RTOL_MIN on the entry points that take it
// (mixed_ok: the direct traces, job tables and servers).
int check_method_precision(const malbec_term& t, malbec_precision prec, bool mixed_ok) {
  if (t.method != MALBEC_METHOD_DOPRI5 || prec == MALBEC_FP64) return MALBEC_OK;
  if (mixed_ok && prec == MALBEC_FP32_MIXED && t.rtol >= MALBEC_DOPRI5_MIXED_RTOL_MIN) return MALBEC_OK;
  return MALBEC_EINVAL;
}

namespace {

struct DeviceInfo {
  int sm_count = 0;
};
std::mutex g_dev_mu;
DeviceInfo g_dev[64];

int device_sms(int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_dev[dev].sm_count == 0) {
    e = cudaDeviceGetAttribute(&g_dev[dev].sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_cuda_error(e);
  }
  *sms = g_dev[dev].sm_count;
  return MALBEC_OK;
}

}  // namespace

namespace {
std::mutex g_launch_mu;
malbec_launch_config g_launch = {0, 0, 0, 0, 0, 0, 0};

malbec_launch_config launch_config() {
  std::lock_guard<std::mutex> lk(g_launch_mu);
  return g_launch;
}
}  // namespace

// Launch shape: persistent warps, as many as fit (occupancy) but no more than
// the rays need; small batches spread one warp per block across the SMs.
int choose_shape(bool kerr, bool mixed, Source src, Sink sink, uint64_t n, LaunchShape* shape, int* refill_min,
                 int form, int method) {
  return choose_shape_cfg(kerr, mixed, src, sink, n, launch_config(), shape, refill_min, form, method);
}

int choose_shape_cfg(bool kerr, bool mixed, Source src, Sink sink, uint64_t n, const malbec_launch_config& cfg,
                     LaunchShape* shape, int* refill_min, int form, int method) {
  int sms = 0;
  int rc = device_sms(&sms);
  if (rc) return rc;
  const uint64_t warps_needed = (n + 31) / 32;
  int tpb = 128;
  if (warps_needed < (uint64_t)sms * 4) tpb = 32;
  if (cfg.threads_per_block) tpb = (int)cfg.threads_per_block;
  // the exchange as launch_trace will decide it: off for whole-image cameras
  // unless asked for
  const bool banks = mixed && method == MALBEC_METHOD_RK4 && (cfg.exchange ? cfg.exchange == 1 : src != kSrcCamera);
  int per_sm = trace_max_blocks_per_sm(kerr, mixed, src, sink, banks, tpb, form, method);
  if (per_sm <= 0) per_sm = 1;
  // Resident warps per SM.  FP64: two per SM sub-partition; the second warp
  // issues while the first waits on an integer test of an FP64 result
  // (1024^2 camera: 135.1 ms against 142.7 with one warp per sub-partition;
  // Dormand-Prince at 1e-9: 311 against 333 ms).  The FP64 unit costs the
  // same per warp instruction whatever the number of active lanes.
  // FP32_MIXED: two per sub-partition, three for whole-image cameras (their
  // kernels are held to 168 registers for it; latency-bound with two: 1024^2
  // render 9.4-9.7 ms against 11.0).
  const int target_warps = mixed ? (src == kSrcCamera ? 12 : 8) : 8;
  int want = target_warps / (tpb / 32);
  if (want < 1) want = 1;
  if (cfg.blocks_per_sm) want = (int)cfg.blocks_per_sm;
  if (want < per_sm) per_sm = want;
  const uint64_t max_blocks = (uint64_t)sms * per_sm;
  const uint64_t blocks_needed = (warps_needed + (tpb / 32) - 1) / (tpb / 32);
  shape->threads_per_block = tpb;
  shape->blocks = (int)(blocks_needed < max_blocks ? blocks_needed : max_blocks);
  // refill granularity.  FP64: a warp waits for 2 dead lanes (the new rays'
  // set-up then runs on two lanes at once; 1024^2 camera: 196.7 ms against
  // 198.0 for 1, 197.0 for 4, 200.9 for 8).  FP32_MIXED cameras: a warp that
  // takes many new rays at once holds neighbouring pixels, which reach their
  // FP64 zones together (zone steps with fuller warps) and share one pass of
  // the FP64 set-up; but it also waits for the slowest of them, which pays
  // only when each lane slot sees many rays.  By rays per resident lane g:
  // 32 for g >= 16, 8 for g >= 4, else 1 (measured, ms: 256^2, g = 1.7:
  // 3.29 / 3.53 / 5.88 for 1 / 8 / 32; 512^2, g = 6.7: 6.54 / 5.64 / 7.72;
  // 1024^2, g = 27: 20.2 / 15.1 / 11.4; 2048^2, g = 108: 70.0 / 50.5 / 42.4).
  // Other FP32_MIXED sources refill every dead lane.
  if (cfg.refill_min) {
    *refill_min = (int)cfg.refill_min;
  } else if (!mixed) {
    *refill_min = 2;
  } else if (src == kSrcCamera) {
    const double g = (double)n / ((double)shape->blocks * (double)shape->threads_per_block);
    *refill_min = g >= 16.0 ? 32 : (g >= 4.0 ? 8 : 1);
  } else {
    *refill_min = 1;
  }
  return MALBEC_OK;
}

namespace {

// Enqueue scratch allocation + zeroing, the trace kernel and the scratch free.
int run_trace(TraceParams& p, bool kerr, bool mixed, Source src, Sink sink, cudaStream_t stream) {
  LaunchShape shape;
  int refill_min = 1;
  int rc = choose_shape(kerr, mixed, src, sink, p.n, &shape, &refill_min, (int)p.form, (int)p.method);
  if (rc) return rc;
  p.refill_min = refill_min;
  fill_zone(p);
  // automatic zone wait for whole-image cameras: 1 warp step.  Their rays
  // meet the FP64 zone near the photon orbits, a few lanes of a warp at a
  // time, and a ray held back for a fuller FP64 batch holds its warp's
  // refill back with it (1024^2 camera, FP32_MIXED: 6.6 ms against 8.2 ms
  // with 64, every pixel's result the same); other sources keep 64.
  if (src == kSrcCamera && launch_config().zone_wait == 0) p.zone_wait = 1;
  void* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, 256, stream);
  if (e != cudaSuccess) return set_cuda_error(e);
  e = cudaMemsetAsync(scratch, 0, 256, stream);
  if (e == cudaSuccess) {
    p.head = static_cast<unsigned long long*>(scratch);
    e = launch_trace(p, kerr, mixed, src, sink, shape, stream);
  }
  cudaError_t e2 = cudaFreeAsync(scratch, stream);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (e2 != cudaSuccess) return set_cuda_error(e2);
  return MALBEC_OK;
}

std::mutex g_zone_mu;
malbec_mixed_zone g_zone = {MALBEC_ZONE_HORIZON_FACTOR, MALBEC_ZONE_PHOTON_MARGIN, MALBEC_ZONE_POLE_SIN};

}  // namespace

void fill_zone(TraceParams& p) {
  {
    std::lock_guard<std::mutex> lk(g_zone_mu);
    p.zone_horizon = g_zone.horizon_factor;
    p.zone_photon = g_zone.photon_margin;
    p.zone_pole = g_zone.pole_sin;
  }
  const malbec_launch_config cfg = launch_config();
  p.zone_batch = cfg.zone_batch ? (int)cfg.zone_batch : -1;  // -1: the launcher decides
  p.zone_wait = cfg.zone_wait ? (int)cfg.zone_wait : 64;
  p.exchange = cfg.exchange ? (cfg.exchange == 1 ? 1 : 0) : -1;  // -1: the launcher decides
  p.zone_wait_ns = (uint64_t)(cfg.zone_wait_limit_us ? cfg.zone_wait_limit_us : 2000000u) * 1000ull;
}

int set_cuda_error(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorString(e);
  return MALBEC_ECUDA;
}

CameraConst make_camera_const(double M, double a, const malbec_camera& c) {
  CameraConst k;
  k.r_obs = c.r_obs;
  k.incl = c.incl;
  k.fov_half = c.fov_half;
  k.nx = c.nx;
  k.ny = c.ny;
  k.so = sin(c.incl);
  k.co = cos(c.incl);
  const double r = c.r_obs, s2 = k.so * k.so;
  const double rho2 = r * r + a * a * k.co * k.co;
  const double Delta = r * r - 2.0 * M * r + a * a;
  const double q = 2.0 * M * r / rho2;
  const double g_tt = q - 1.0, g_tp = -a * s2 * q, g_pp = s2 * (r * r + a * a + a * a * s2 * q);
  const double det = -Delta * s2;
  k.Delta_o = Delta;
  k.r2a2_o = r * r + a * a;
  k.gtt = g_pp / det;
  k.gtp = -g_tp / det;
  k.gpp = g_tt / det;
  k.grr = Delta / rho2;
  k.ghh = 1.0 / rho2;
  return k;
}

}  // namespace malbec

using namespace malbec;

extern "C" {

const char* malbec_strerror(int code) {
  switch (code) {
    case MALBEC_OK: return "ok";
    case MALBEC_EINVAL: return "invalid argument";
    case MALBEC_ENOMEM: return "out of memory or over the HBM budget";
    case MALBEC_EBUSY: return "admission queue full";
    case MALBEC_ETIMEDOUT: return "bounded device wait timed out";
    case MALBEC_ECUDA: return "CUDA runtime error";
    case MALBEC_ENOTFOUND: return "unknown job";
    case MALBEC_ESCRATCH: return "needs more scratch than the static no-allocation block holds";
    default: return "unknown error code";
  }
}

const char* malbec_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int malbec_set_mixed_zone(const malbec_mixed_zone* z) {
  malbec_mixed_zone v = {MALBEC_ZONE_HORIZON_FACTOR, MALBEC_ZONE_PHOTON_MARGIN, MALBEC_ZONE_POLE_SIN};
  if (z) {
    if (!isfinite(z->horizon_factor) || z->horizon_factor < 1.0 || !isfinite(z->photon_margin) ||
        z->photon_margin < 0.0 || !(z->pole_sin >= 0.0 && z->pole_sin <= 1.0))
      return MALBEC_EINVAL;
    v = *z;
  }
  std::lock_guard<std::mutex> lk(g_zone_mu);
  g_zone = v;
  return MALBEC_OK;
}

int malbec_set_launch_config(const malbec_launch_config* cfg) {
  malbec_launch_config v = {0, 0, 0, 0, 0, 0, 0};
  if (cfg) {
    if (cfg->threads_per_block && (cfg->threads_per_block % 32 != 0 || cfg->threads_per_block > 256))
      return MALBEC_EINVAL;
    if (cfg->blocks_per_sm > 64 || cfg->refill_min > 32 || cfg->zone_batch > 32 || cfg->zone_wait > 1000000 ||
        cfg->exchange > 2)
      return MALBEC_EINVAL;
    v = *cfg;
  }
  std::lock_guard<std::mutex> lk(g_launch_mu);
  g_launch = v;
  return MALBEC_OK;
}

int malbec_get_launch_config(malbec_launch_config* cfg) {
  if (!cfg) return MALBEC_EINVAL;
  *cfg = launch_config();
  return MALBEC_OK;
}

int malbec_get_mixed_zone(malbec_mixed_zone* z) {
  if (!z) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(g_zone_mu);
  *z = g_zone;
  return MALBEC_OK;
}

int malbec_out_layout(malbec_out_mode mode, malbec_precision prec, uint64_t n, uint32_t n_steps_cap,
                      uint32_t stride, malbec_layout* L) {
  if (!L || n == 0) return MALBEC_EINVAL;
  if (mode != MALBEC_OUT_FINAL && mode != MALBEC_OUT_STRIDED && mode != MALBEC_OUT_STRIDED_CARTESIAN)
    return MALBEC_EINVAL;
  if (prec != MALBEC_FP64 && prec != MALBEC_FP32_MIXED) return MALBEC_EINVAL;
  const bool strided = mode != MALBEC_OUT_FINAL;
  if (strided && stride == 0) return MALBEC_EINVAL;
  if (n > (1ull << 40)) return MALBEC_EINVAL;
  size_t off = 0;
  L->y = off;
  off = align256(off + 8 * n * sizeof(double));
  L->lambda = off;
  off = align256(off + n * sizeof(double));
  L->inv0 = off;
  off = align256(off + 4 * n * sizeof(double));
  L->inv1 = off;
  off = align256(off + 4 * n * sizeof(double));
  L->steps = off;
  off = align256(off + n * sizeof(uint32_t));
  L->fate = off;
  off = align256(off + n);
  L->traj = 0;
  L->n_samples = 0;
  if (strided) {
    const uint64_t ns = (uint64_t)(n_steps_cap / stride) + 1;
    const size_t elem = prec == MALBEC_FP64 ? sizeof(double) : sizeof(float);
    const size_t comps = mode == MALBEC_OUT_STRIDED_CARTESIAN ? 4 : 8;
    const long double bytes = (long double)n * ns * comps * elem;
    if (bytes > 2.0e14L) return MALBEC_EINVAL;  // beyond any device memory
    L->traj = off;
    L->n_samples = ns;
    off = align256(off + (size_t)(n * ns * comps * elem));
  }
  L->total = off;
  return MALBEC_OK;
}

size_t malbec_out_bytes(malbec_out_mode mode, malbec_precision prec, uint64_t n, uint32_t n_steps_cap,
                        uint32_t stride) {
  malbec_layout L;
  if (malbec_out_layout(mode, prec, n, n_steps_cap, stride, &L) != MALBEC_OK) return 0;
  return L.total;
}

int malbec_trace(malbec_metric m, const double* ics, uint64_t n, malbec_term t, malbec_out_mode mode,
                 uint32_t stride, malbec_precision prec, void* out, malbec_stream stream) {
  int rc = check_metric(m);
  if (rc) return rc;
  rc = check_term(t, m);
  if (rc) return rc;
  rc = check_method_precision(t, prec, true);
  if (rc) return rc;
  if (!ics || !out) return MALBEC_EINVAL;
  malbec_layout L;
  rc = malbec_out_layout(mode, prec, n, t.n_steps_cap, stride, &L);
  if (rc) return rc;
  if (((uintptr_t)out & 255u) != 0) return MALBEC_EINVAL;
  char* o = static_cast<char*>(out);
  TraceParams p;
  memset(&p, 0, sizeof(p));
  p.M = m.M;
  p.a = m.a;
  p.a_per_ray = m.a_per_ray;
  p.eps_hor = t.eps_hor;
  p.r_esc = t.r_esc;
  p.dl = t.dl;
  p.dl_r_scale = t.dl_r_scale;
  p.form = t.form;
  p.method = t.method;
  p.rtol = t.rtol;
  p.atol = t.atol;
  p.cap = t.n_steps_cap;
  p.ics = ics;
  p.n = n;
  p.y_out = reinterpret_cast<double*>(o + L.y);
  p.lambda_out = reinterpret_cast<double*>(o + L.lambda);
  p.inv0_out = reinterpret_cast<double*>(o + L.inv0);
  p.inv1_out = reinterpret_cast<double*>(o + L.inv1);
  p.steps_out = reinterpret_cast<uint32_t*>(o + L.steps);
  p.fate_out = reinterpret_cast<uint8_t*>(o + L.fate);
  const bool strided = mode != MALBEC_OUT_FINAL;
  p.traj = strided ? static_cast<void*>(o + L.traj) : nullptr;
  p.stride = strided ? stride : 1;
  p.n_samples = L.n_samples;
  p.traj_cartesian = mode == MALBEC_OUT_STRIDED_CARTESIAN ? 1 : 0;
  const bool kerr = !(m.a == 0.0 && m.a_per_ray == nullptr);
  return run_trace(p, kerr, prec == MALBEC_FP32_MIXED, kSrcStates, strided ? kSinkStrided : kSinkFinal,
                   (cudaStream_t)stream);
}

int malbec_camera_out_layout(const malbec_camera* cam, malbec_camera_layout* L) {
  if (!cam || !L || cam->nx == 0 || cam->ny == 0) return MALBEC_EINVAL;
  const uint64_t n = (uint64_t)cam->nx * cam->ny;
  size_t off = 0;
  L->fate = off;
  off = align256(off + n);
  L->steps = off;
  off = align256(off + n * sizeof(uint32_t));
  L->theta = off;
  off = align256(off + n * sizeof(double));
  L->phi = off;
  off = align256(off + n * sizeof(double));
  L->total = off;
  return MALBEC_OK;
}

static int check_camera(const malbec_metric& m, const malbec_camera* cam, const malbec_term* t) {
  if (!cam || m.a_per_ray) return MALBEC_EINVAL;
  if (cam->nx == 0 || cam->ny == 0) return MALBEC_EINVAL;
  if (!finite_pos(cam->fov_half) || !isfinite(cam->incl) || !(cam->incl > 0.0) || !(cam->incl < M_PI))
    return MALBEC_EINVAL;
  const double rp = host_r_plus(m.M, m.a);
  const double eps = t ? t->eps_hor : 0.0;
  if (!isfinite(cam->r_obs) || !(cam->r_obs > (1.0 + eps) * rp)) return MALBEC_EINVAL;
  if (t && !(cam->r_obs < t->r_esc)) return MALBEC_EINVAL;
  return MALBEC_OK;
}

}  // extern "C"

int malbec::check_camera_desc(const malbec_metric& m, const malbec_camera* cam, const malbec_term* t) {
  return check_camera(m, cam, t);
}

extern "C" {

int malbec_trace_camera(malbec_metric m, const malbec_camera* cam, malbec_term t, malbec_precision prec, void* out,
                        malbec_stream stream) {
  int rc = check_metric(m);
  if (rc) return rc;
  rc = check_term(t, m);
  if (rc) return rc;
  rc = check_camera(m, cam, &t);
  if (rc) return rc;
  if (!out || ((uintptr_t)out & 255u) != 0) return MALBEC_EINVAL;
  if (prec != MALBEC_FP64 && prec != MALBEC_FP32_MIXED) return MALBEC_EINVAL;
  rc = check_method_precision(t, prec, true);
  if (rc) return rc;
  malbec_camera_layout L;
  rc = malbec_camera_out_layout(cam, &L);
  if (rc) return rc;
  char* o = static_cast<char*>(out);
  TraceParams p;
  memset(&p, 0, sizeof(p));
  p.M = m.M;
  p.a = m.a;
  p.eps_hor = t.eps_hor;
  p.r_esc = t.r_esc;
  p.dl = t.dl;
  p.dl_r_scale = t.dl_r_scale;
  p.form = t.form;
  p.method = t.method;
  p.rtol = t.rtol;
  p.atol = t.atol;
  p.cap = t.n_steps_cap;
  p.n = (uint64_t)cam->nx * cam->ny;
  p.cam = make_camera_const(m.M, m.a, *cam);
  p.fate_out = reinterpret_cast<uint8_t*>(o + L.fate);
  p.steps_out = reinterpret_cast<uint32_t*>(o + L.steps);
  p.theta_out = reinterpret_cast<double*>(o + L.theta);
  p.phi_out = reinterpret_cast<double*>(o + L.phi);
  p.stride = 1;
  const bool kerr = m.a != 0.0;
  return run_trace(p, kerr, prec == MALBEC_FP32_MIXED, kSrcCamera, kSinkCamera, (cudaStream_t)stream);
}

int malbec_ic_camera(malbec_metric m, const malbec_camera* cam, const uint64_t* pixels, uint64_t n, double* ics,
                     malbec_stream stream) {
  int rc = check_metric(m);
  if (rc) return rc;
  rc = check_camera(m, cam, nullptr);
  if (rc) return rc;
  if (!pixels || !ics || n == 0) return MALBEC_EINVAL;
  cudaError_t e = launch_ic_camera(m.M, m.a, make_camera_const(m.M, m.a, *cam), pixels, n, ics, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int malbec_ic_circular(malbec_metric m, const double* radii, uint64_t n, int prograde, double* ics,
                       malbec_stream stream) {
  int rc = check_metric(m);
  if (rc) return rc;
  if (m.a_per_ray || !radii || !ics || n == 0) return MALBEC_EINVAL;
  cudaError_t e = launch_ic_circular(m.M, m.a, radii, n, prograde, ics, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int malbec_ic_bound(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t index0, uint64_t n, double* ics,
                    double* spins, int32_t* accepted, malbec_stream stream) {
  if (!finite_pos(M) || !isfinite(a_max) || a_max < 0.0 || !(a_max < M)) return MALBEC_EINVAL;
  if (!ics || !spins || !accepted || n == 0) return MALBEC_EINVAL;
  if (index0 + n < index0 || index0 + n > (1ull << 55)) return MALBEC_EINVAL;  // counters index*256 fit in 64 bits
  cudaError_t e = launch_ic_bound(M, a_max, spin_fixed, seed, index0, n, ics, spins, accepted, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int malbec_invariants(malbec_metric m, const double* states, uint64_t n, double* inv, malbec_stream stream) {
  int rc = check_metric(m);
  if (rc) return rc;
  if (!states || !inv || n == 0) return MALBEC_EINVAL;
  cudaError_t e = launch_invariants(m.M, m.a, m.a_per_ray, states, n, inv, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int malbec_ic_from_paper(malbec_metric m, const double* rows, uint64_t n, double* ics, malbec_stream stream) {
  int rc = check_metric(m);
  if (rc) return rc;
  if (!rows || !ics || n == 0 || rows == ics) return MALBEC_EINVAL;
  cudaError_t e = launch_ic_from_paper(m.M, m.a, m.a_per_ray, rows, n, ics, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int malbec_wait_status(uint64_t* timeouts) {
  static std::mutex mu;
  static unsigned long long seen[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return MALBEC_EINVAL;
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return set_cuda_error(e);
  unsigned long long total = 0;
  e = read_wait_timeouts(&total);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (timeouts) *timeouts = total;
  std::lock_guard<std::mutex> lk(mu);
  const bool grew = total > seen[dev];
  seen[dev] = total;
  return grew ? MALBEC_ETIMEDOUT : MALBEC_OK;
}

const char* malbec_build_info(void) {
#define MALBEC_S2(x) #x
#define MALBEC_S(x) MALBEC_S2(x)
  return "libmalbec: sm_103a, nvcc " MALBEC_S(__CUDACC_VER_MAJOR__) "." MALBEC_S(__CUDACC_VER_MINOR__) ", -O3, no fast-math, no implicit FMA contraction (explicit fma only)";
}

}  // extern "C"

// trace_kernel.cuh -- the persistent work-queue geodesic kernel (instantiated
// by trace.cu and trace_dopri.cu).
//
// One ray per lane.  Warps stay resident and pull ray indices from a device
// counter: after every RK4 step each lane tests its ray for termination
// (capture at (1+eps) r_+, escape, non-finite, step cap; the paper's
// per-thread horizon stop, Sec. 5), a warp ballot counts idle lanes, and once
// at least `refill_min` lanes are idle the warp takes that many new rays with
// a single atomicAdd and hands them to the idle lanes.  Rays therefore never
// share a lane's time with a long-running neighbour; results do not depend on
// which lane or warp ran a ray.
//
// Precision: FP64 (every operation in double), or FP32_MIXED: the state is
// kept as a compensated pair (hi, lo) of floats, the RHS and RK4 stages run in
// FP32, and the increments h/6 (k1 + 2k2 + 2k3 + k4) -- with h/6 as a float
// pair -- are added with TwoSum.  lambda is accumulated in FP64 (the h of
// FP32 steps through an error-free float-pair partial sum flushed every 32
// steps) and the invariants are evaluated in FP64 (the end norm of an
// FP32_MIXED camera pixel in FP32, for its validity flag); a step whose start lies
// inside the FP64 zone (near the horizon, near the photon orbits for null
// rays, or near the polar axis where the BL Christoffel symbols diverge) runs
// entirely in FP64, and the warps of a block exchange rays so that zone steps
// run with full warps (see the block banks below).  On a part whose FP64 rate
// is 1/64 of its FP32 rate every FP64 operation in the bulk path counts: an
// FP32 step has none.  FP32 steps test termination on the hi words against
// the thresholds rounded to float.
#pragma once
#include <math.h>

#include "bound.cuh"
#include "camera.cuh"
#include "geodesic.cuh"
#include "fp32pair.cuh"
#include "internal.h"

namespace malbec {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxTPB = 256;

__device__ __forceinline__ double dev_r_plus(double M, double a) { return M + sqrt(fma(-a, a, M * M)); }

// Retrograde circular photon orbit 2M (1 + cos(2/3 arccos(a/M))).
__device__ __forceinline__ double dev_r_photon_retro(double M, double a) {
  return 2.0 * M * (1.0 + cos((2.0 / 3.0) * acos(a / M)));
}

// Non-finite test on the exponent bits (integer pipe, no FP64 compare).
__device__ __forceinline__ bool finite8(const double y[8]) {
  int bad = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) bad |= ((__double2hiint(y[c]) & 0x7ff00000) == 0x7ff00000);
  return !bad;
}
__device__ __forceinline__ bool finite8f(const float y[8]) {
  int bad = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) bad |= ((__float_as_int(y[c]) & 0x7f800000) == 0x7f800000);
  return !bad;
}

// g(u,u) of an FP32 state in FP32 arithmetic, Kerr in BL coordinates: the
// geodesic form from (x, u) as g_ab u^a u^b, the canonical forms from (x, p)
// as g^ab p_a p_b (the inverse (t, phi) block has det -Delta sin^2).
template <bool kCanon>
__device__ __forceinline__ float state_norm_f(float M, float a, const float y[8]) {
  float s, c;
  sincosf(y[2], &s, &c);
  const float r = y[1], a2 = a * a, s2 = s * s;
  const float rho2 = fmaf(a2, c * c, r * r);
  const float Delta = fmaf(r, r - 2.0f * M, a2);
  const float q = 2.0f * M * r / rho2;
  const float gtt = q - 1.0f;
  const float gtp = -a * s2 * q;
  const float gpp = s2 * fmaf(a2 * s2, q, fmaf(r, r, a2));
  if constexpr (kCanon) {
    const float det = -Delta * s2;
    const float ut = fmaf(gpp, y[4], -gtp * y[7]) / det;
    const float up = fmaf(gtt, y[7], -gtp * y[4]) / det;
    return fmaf(y[4], ut, fmaf(Delta / rho2 * y[5], y[5], fmaf(y[6] / rho2, y[6], y[7] * up)));
  } else {
    const float pt = fmaf(gtt, y[4], gtp * y[7]);
    const float pp = fmaf(gtp, y[4], gpp * y[7]);
    return fmaf(pt, y[4], fmaf(rho2 / Delta * y[5], y[5], fmaf(rho2 * y[6], y[6], pp * y[7])));
  }
}

// Trajectory sample k of ray id: the state (8 components), or with
// p.traj_cartesian the paper's output record (t, x, y, z) of eq. coord,
// x = sqrt(r^2 + a^2) sin th cos ph, y = sqrt(r^2 + a^2) sin th sin ph,
// z = r cos th.  FP32_MIXED samples come from the hi words, in FP32.
template <bool kMixed>
__device__ __forceinline__ void store_sample(const TraceParams& p, double a, uint64_t id, uint64_t k,
                                             const double y[8], const float hi[8]) {
  if (p.traj_cartesian) {
    const size_t off = ((size_t)id * p.n_samples + k) * 4;
    if (kMixed) {
      float st, ct, sp, cp;
      sincosf(hi[2], &st, &ct);
      sincosf(hi[3], &sp, &cp);
      const float R = sqrtf(fmaf(hi[1], hi[1], (float)(a * a)));
      *reinterpret_cast<float4*>(static_cast<float*>(p.traj) + off) =
          make_float4(hi[0], R * st * cp, R * st * sp, hi[1] * ct);
    } else {
      double st, ct, sp, cp;
      sincos(y[2], &st, &ct);
      sincos(y[3], &sp, &cp);
      const double R = sqrt(fma(y[1], y[1], a * a));
      double2* t = reinterpret_cast<double2*>(static_cast<double*>(p.traj) + off);
      t[0] = make_double2(y[0], R * st * cp);
      t[1] = make_double2(R * st * sp, y[1] * ct);
    }
    return;
  }
  const size_t off = ((size_t)id * p.n_samples + k) * 8;
  if (kMixed) {
    float4* t = reinterpret_cast<float4*>(static_cast<float*>(p.traj) + off);
    t[0] = make_float4(hi[0], hi[1], hi[2], hi[3]);
    t[1] = make_float4(hi[4], hi[5], hi[6], hi[7]);
  } else {
    double2* t = reinterpret_cast<double2*>(static_cast<double*>(p.traj) + off);
#pragma unroll
    for (int c = 0; c < 4; ++c) t[c] = make_double2(y[2 * c], y[2 * c + 1]);
  }
}

template <bool kMixed>
__device__ __forceinline__ void store_nan_samples(const TraceParams& p, uint64_t id, uint64_t k0) {
  const int comps = p.traj_cartesian ? 4 : 8;
  for (uint64_t k = k0; k < p.n_samples; ++k) {
    const size_t off = ((size_t)id * p.n_samples + k) * comps;
    if (kMixed) {
      const float fn = __int_as_float(0x7fc00000);
      float4* t = reinterpret_cast<float4*>(static_cast<float*>(p.traj) + off);
      for (int c = 0; c < comps / 4; ++c) t[c] = make_float4(fn, fn, fn, fn);
    } else {
      const double qn = __longlong_as_double(0x7ff8000000000000ll);
      double2* t = reinterpret_cast<double2*>(static_cast<double*>(p.traj) + off);
      for (int c = 0; c < comps / 2; ++c) t[c] = make_double2(qn, qn);
    }
  }
}

// One FP32 RK4 step on the compensated state (hi, lo).  The stage points are
// hi + (lo + c h k), so the low words enter the right-hand side; the
// increments h/6 (k1 + 2k2 + 2k3 + k4) use h/6 as a float pair (h6h, h6l) and
// are added with TwoSum.  One copy of the right-hand side (stage loop not
// unrolled).  The component-wise parts (the stage velocities, the weighted
// sums, the compensated update of the eight components) run as paired FP32
// operations on two components at once (the FP32_MIXED camera is
// issue-bound: 8.6 -> 8.2 ms per 1024^2 render, the same image bit for
// bit).  Returns the smallest stage radius.
template <bool kKerr>
__device__ __forceinline__ float rk4_step_mixed(const BH<float>& bh, float hf, float h6h, float h6l, float hi[8],
                                                float lo[8]) {
  const float hh = 0.5f * hf;
  float r = hi[1], th = hi[2];
  float2 u01 = make_float2(hi[4], hi[5]), u23 = make_float2(hi[6], hi[7]);
  const float2 hi45 = make_float2(hi[4], hi[5]), hi67 = make_float2(hi[6], hi[7]);
  const float2 lo45 = make_float2(lo[4], lo[5]), lo67 = make_float2(lo[6], lo[7]);
  float2 sx01, sx23, su01, su23;
  float rmin = 0.f;
#pragma unroll 1
  for (int s = 0; s < 4; ++s) {
    float acc[4];
    accel<kKerr, float>(bh, r, th, u01.x, u01.y, u23.x, u23.y, acc);
    const float2 a01 = make_float2(acc[0], acc[1]), a23 = make_float2(acc[2], acc[3]);
    if (s == 0) {
      sx01 = u01;
      sx23 = u23;
      su01 = a01;
      su23 = a23;
    } else {
      const float w = s == 3 ? 1.f : 2.f;
      const float2 w2 = make_float2(w, w);
      sx01 = f2fma(w2, u01, sx01);
      sx23 = f2fma(w2, u23, sx23);
      su01 = f2fma(w2, a01, su01);
      su23 = f2fma(w2, a23, su23);
    }
    if (s < 3) {
      const float c = s < 2 ? hh : hf;
      const float2 c2 = make_float2(c, c);
      r = hi[1] + fmaf(c, u01.y, lo[1]);
      th = hi[2] + fmaf(c, u23.x, lo[2]);
      u01 = f2add(hi45, f2fma(c2, a01, lo45));
      u23 = f2add(hi67, f2fma(c2, a23, lo67));
      rmin = s == 0 ? r : fminf(rmin, r);
    }
  }
  const float2 H = make_float2(h6h, h6h), L = make_float2(h6l, h6l);
  float2 sxp[2] = {sx01, sx23}, sup[2] = {su01, su23};
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float2 dx = f2mul(H, sxp[k]);
    const float2 dxe = f2fma(L, sxp[k], f2fma(H, sxp[k], make_float2(-dx.x, -dx.y)));
    const float2 du = f2mul(H, sup[k]);
    const float2 due = f2fma(L, sup[k], f2fma(H, sup[k], make_float2(-du.x, -du.y)));
    float2 h0 = make_float2(hi[2 * k], hi[2 * k + 1]), l0 = make_float2(lo[2 * k], lo[2 * k + 1]);
    float2 h1 = make_float2(hi[4 + 2 * k], hi[5 + 2 * k]), l1 = make_float2(lo[4 + 2 * k], lo[5 + 2 * k]);
    comp_add2(h0, l0, dx, dxe);
    comp_add2(h1, l1, du, due);
    hi[2 * k] = h0.x;
    hi[2 * k + 1] = h0.y;
    lo[2 * k] = l0.x;
    lo[2 * k + 1] = l0.y;
    hi[4 + 2 * k] = h1.x;
    hi[5 + 2 * k] = h1.y;
    lo[4 + 2 * k] = l1.x;
    lo[5 + 2 * k] = l1.y;
  }
  return rmin;
}

// The canonical forms of rk4_step_mixed: z = (x, p) as compensated pairs,
// p_t = z[4] and p_ph = z[7] fixed (their float hi words enter the right-hand
// side); t, r, theta, phi, p_r, p_theta are integrated.
template <int kForm>
__device__ __forceinline__ float rk4_step_mixed_ham(const BH<float>& bh, float hf, float h6h, float h6l, float hi[8],
                                                    float lo[8]) {
  const float hh = 0.5f * hf;
  float2 rth = make_float2(hi[1], hi[2]), pp = make_float2(hi[5], hi[6]);  // (r, theta), (p_r, p_theta)
  const float2 hi12 = rth, hi56 = pp;
  const float2 lo12 = make_float2(lo[1], lo[2]), lo56 = make_float2(lo[5], lo[6]);
  float2 sx[3];  // (t, r), (theta, phi), (p_r, p_theta)
  float rmin = 0.f;
#pragma unroll 1
  for (int s = 0; s < 4; ++s) {
    float f[6];
    ham_rhs<kForm, float>(bh, rth.x, rth.y, hi[4], pp.x, pp.y, hi[7], f);
    const float2 f01 = make_float2(f[0], f[1]), f23 = make_float2(f[2], f[3]), f45 = make_float2(f[4], f[5]);
    if (s == 0) {
      sx[0] = f01;
      sx[1] = f23;
      sx[2] = f45;
    } else {
      const float w = s == 3 ? 1.f : 2.f;
      const float2 w2 = make_float2(w, w);
      sx[0] = f2fma(w2, f01, sx[0]);
      sx[1] = f2fma(w2, f23, sx[1]);
      sx[2] = f2fma(w2, f45, sx[2]);
    }
    if (s < 3) {
      const float c = s < 2 ? hh : hf;
      const float2 c2 = make_float2(c, c);
      rth = f2add(hi12, f2fma(c2, make_float2(f[1], f[2]), lo12));
      pp = f2add(hi56, f2fma(c2, f45, lo56));
      rmin = s == 0 ? rth.x : fminf(rmin, rth.x);
    }
  }
  const float2 H = make_float2(h6h, h6h), L = make_float2(h6l, h6l);
  const int comp[3] = {0, 2, 5};  // first component of each pair
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int j = comp[k];
    const float2 d = f2mul(H, sx[k]);
    const float2 de = f2fma(L, sx[k], f2fma(H, sx[k], make_float2(-d.x, -d.y)));
    float2 h = make_float2(hi[j], hi[j + 1]), l = make_float2(lo[j], lo[j + 1]);
    comp_add2(h, l, d, de);
    hi[j] = h.x;
    hi[j + 1] = h.y;
    lo[j] = l.x;
    lo[j + 1] = l.y;
  }
  return rmin;
}

// FP32_MIXED Dormand-Prince 5(4): one attempt of size hf in FP32 on the
// compensated state (hi, lo), with the tableau of dopri5_attempt.  Stage
// points are hi + (lo + hf d), d = sum_j a_ij k_j; k1 is the first stage
// (the last accepted attempt's k7).  Out: the fifth-order increment as a
// float pair (dx, dxe: hf times the b-weighted sum and that product's
// rounding error), the embedded error estimate e = hf sum_j (b_j - bhat_j) k_j
// and k7 = f at the fifth-order point.  Canonical forms: p_t = hi[4] and
// p_ph = hi[7] are fixed (their k components are 0).  Returns the smallest
// stage radius among the stage points 2..7.

// The FP32_MIXED Dormand-Prince kernels call one out-of-line copy of each
// right-hand side (and of the FP64 zone attempt) instead of inlining seven:
// the inlined kernel stalled on instruction fetch (ncu: no_instruction 3.6
// per issue, 25% of issue slots used); 1024^2 camera at rtol 1e-6: 17.1 ->
// 15.2 ms, the same arithmetic.
template <bool kKerr>
__device__ __noinline__ void accel_f32_call(const BH<float>& bh, float r, float th, float ut, float ur, float uth,
                                            float uph, float* acc) {
  accel<kKerr, float>(bh, r, th, ut, ur, uth, uph, acc);
}
template <int kForm>
__device__ __noinline__ void ham_f32_call(const BH<float>& bh, float r, float th, float pt, float pr, float pth,
                                          float pph, float* f) {
  ham_rhs<kForm, float>(bh, r, th, pt, pr, pth, pph, f);
}
template <bool kKerr, int kForm>
__device__ __noinline__ double dopri5_attempt_call(const BH<double>& bh, double h, const double* y, const double* k1,
                                                   double* y5, double* e, double* k7) {
  return dopri5_attempt<kKerr, kForm>(bh, h, y, k1, y5, e, k7);
}
template <bool kKerr, int kForm>
__device__ __forceinline__ float dopri5_attempt_mixed(const BH<float>& bh, float hf, const float hi[8],
                                                      const float lo[8], const float k1[8], float dx[8],
                                                      float dxe[8], float e[8], float k7[8]) {
  float k2[8], k3[8], k4[8], k5[8], k6[8];
  float d[8];
  float rmin = 0.f;
  auto stage = [&](float k[8], bool first) {
    float z[8];
#pragma unroll
    for (int c = 1; c < 8; ++c) z[c] = hi[c] + fmaf(hf, d[c], lo[c]);
    if constexpr (kForm == MALBEC_FORM_GEODESIC) {
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = z[4 + j];
      accel_f32_call<kKerr>(bh, z[1], z[2], z[4], z[5], z[6], z[7], k + 4);
    } else {
      float f[6];
      ham_f32_call<kForm>(bh, z[1], z[2], hi[4], z[5], z[6], hi[7], f);
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = f[j];
      k[4] = 0.f;
      k[5] = f[4];
      k[6] = f[5];
      k[7] = 0.f;
    }
    rmin = first ? z[1] : fminf(rmin, z[1]);
  };
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = (1.0f / 5.0f) * k1[q];
  stage(k2, true);
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = fmaf(3.0f / 40.0f, k1[q], (9.0f / 40.0f) * k2[q]);
  stage(k3, false);
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = fmaf(44.0f / 45.0f, k1[q], fmaf(-56.0f / 15.0f, k2[q], (32.0f / 9.0f) * k3[q]));
  stage(k4, false);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    d[q] = fmaf(19372.0f / 6561.0f, k1[q],
                fmaf(-25360.0f / 2187.0f, k2[q], fmaf(64448.0f / 6561.0f, k3[q], (-212.0f / 729.0f) * k4[q])));
  stage(k5, false);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    d[q] = fmaf(9017.0f / 3168.0f, k1[q],
                fmaf(-355.0f / 33.0f, k2[q],
                     fmaf(46732.0f / 5247.0f, k3[q], fmaf(49.0f / 176.0f, k4[q], (-5103.0f / 18656.0f) * k5[q]))));
  stage(k6, false);
  // the fifth-order weights (a_2 = 0)
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    d[q] = fmaf(35.0f / 384.0f, k1[q],
                fmaf(500.0f / 1113.0f, k3[q],
                     fmaf(125.0f / 192.0f, k4[q], fmaf(-2187.0f / 6784.0f, k5[q], (11.0f / 84.0f) * k6[q]))));
    dx[q] = hf * d[q];
    dxe[q] = fmaf(hf, d[q], -dx[q]);
  }
  stage(k7, false);
  // e = h sum_j (b_j - bhat_j) k_j
#pragma unroll
  for (int q = 0; q < 8; ++q)
    e[q] = hf * fmaf(71.0f / 57600.0f, k1[q],
                     fmaf(-71.0f / 16695.0f, k3[q],
                          fmaf(71.0f / 1920.0f, k4[q],
                               fmaf(-17253.0f / 339200.0f, k5[q], fmaf(22.0f / 525.0f, k6[q], (-1.0f / 40.0f) * k7[q])))));
  return rmin;
}

// dopri5_norm and dopri5_factor in FP32 (the same rule; the error estimate of
// an FP32 attempt carries rounding noise of ~1e-7 of the state, so FP32_MIXED
// runs the method at tolerances rtol >= MALBEC_DOPRI5_MIXED_RTOL_MIN).
__device__ __forceinline__ float dopri5_norm_f(const float y[8], const float y5[8], const float e[8], float rtol,
                                               float atol) {
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float t = e[q] / fmaf(rtol, fmaxf(fabsf(y[q]), fabsf(y5[q])), atol);
    s = fmaf(t, t, s);
  }
  return sqrtf(0.125f * s);
}
__device__ __forceinline__ float dopri5_factor_f(float err, bool accepted, bool after_reject) {
  float q = err > 0.f ? 4.0f * log2f(0.9f) - 0.8f * log2f(err) : 13.0f;
  const float jmax = accepted ? (after_reject ? 0.0f : 13.0f) : -1.0f;
  q = fmaxf(fminf(q, jmax), -10.0f);
  const int j = (int)floorf(q);
  const int r = j & 3;        // j mod 4
  const int ex = (j - r) / 4;  // floor(j / 4)
  const float quarter = r == 0 ? 1.0f : (r == 1 ? 1.18920712f : (r == 2 ? 1.41421356f : 1.68179283f));
  return ldexpf(quarter, ex);
}

__device__ __forceinline__ void step_consts(double dl, double dl_scale, double r_esc, float& h_fix, float& h6h,
                                            float& h6l, float& scale_f, float& r_esc_f) {
  h_fix = (float)dl;
  const double h6 = dl / 6.0;
  h6h = (float)h6;
  h6l = (float)(h6 - (double)h6h);
  scale_f = (float)dl_scale;
  r_esc_f = (float)r_esc;
}

// A job descriptor read around L1 (its slot may have been rewritten by the
// host since this SM last looked at it).
__device__ __forceinline__ JobDesc load_job(const JobDesc* src) {
  JobDesc d;
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* t = reinterpret_cast<unsigned long long*>(&d);
#pragma unroll
  for (int k = 0; k < (int)(sizeof(JobDesc) / 8); ++k) t[k] = __ldcg(s + k);
  return d;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void split_pair(const double y[8], float hi[8], float lo[8]) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    hi[c] = (float)y[c];
    lo[c] = (float)(y[c] - (double)hi[c]);
  }
}

// ---------------------------------------------------------------------------
// FP32_MIXED: exchange of rays between the warps of a block.
//
// The FP64 unit costs the same per warp instruction whatever the number of
// active lanes, and few rays of a warp are in the FP64 zone at a time, so
// zone steps taken where the rays happen to be run with a handful of lanes.
// One warp of each block (the zone warp) therefore collects them: the other
// warps hand a zone ray that would otherwise wait (fewer than zone_batch
// zone lanes in the warp) to the block's zone bank, and take rays the zone
// warp has handed back to the FP32 bank into idle lanes before they claim new
// ones; the zone warp fills its idle lanes from the zone bank and hands its
// FP32 rays to the FP32 bank while zone rays wait.  A ray carries its whole
// state; where it runs changes when its steps run, never their arithmetic.
// Every bank operation holds the block's lock (a bounded try: a warp that
// does not get it simply skips the exchange this time).
constexpr int kBankSlots = 32;

struct RayBank {
  float hi[8][kBankSlots], lo[8][kBankSlots];
  double lam[kBankSlots], M[kBankSlots], a[kBankSlots], dl[kBankSlots], dls[kBankSlots], r_esc[kBankSlots],
      r_cap[kBankSlots];
  unsigned long long id[kBankSlots];
  uint32_t job[kBankSlots], nst[kBankSlots], cap[kBankSlots];
  float r_zone[kBankSlots], pole[kBankSlots], lam_h[kBankSlots], lam_l[kBankSlots];
  uint32_t lam_fix[kBankSlots];
  double n0[kBankSlots], drift_lim[kBankSlots];
};

struct BlockBanks {
  RayBank zone, fp32;
  int n_zone, n_fp32;  // records [0, n) of each bank are valid
  int lock;
  int open;            // the zone warp still takes zone rays
  int alive;           // warps of the block other than the zone warp still running
};
struct NoBanks {
  int unused;
};
template <bool kMixed>
struct BanksFor {
  using type = NoBanks;
};
template <>
struct BanksFor<true> {
  using type = BlockBanks;
};

// ---------------------------------------------------------------------------
// FP64 whole-image cameras: ray starts and ends staged per warp.
//
// The FP64 work at a ray's start (the pixel's initial state, its invariants,
// the canonical momenta) and at its end (the invariants behind the validity
// flag) costs one FP64 warp instruction per operation whether one lane needs
// it or 32, and an FP64 warp refills its lanes a few at a time.  So the warp
// prepares the starts of up to 32 queued pixels at once, one per lane, and
// hands them out as lanes fall idle; and it parks ended rays here and
// finishes up to 32 of them at once.  Each ray's arithmetic is unchanged;
// only when, and in which lane, it runs.  (FP32_MIXED camera warps refill all
// 32 lanes at once, so their starts are batched already.)
struct WarpStage {
  double y0[8][32];          // start states (canonical forms: (x, p))
  double n0[32], dlim0[32];  // norm at the start, drift limit of the flag
  unsigned long long id0[32];
  double y1[7][32];          // end states y[1..7]
  double n1[32], dlim1[32];
  unsigned long long id1[32];
  uint32_t nst1[32], fate1[32];
};
struct NoStage {
  int unused;
};
template <bool kOn>
struct StageFor {
  using type = NoStage;
};
template <>
struct StageFor<true> {
  using type = WarpStage[kMaxTPB / 32];
};
static_assert(sizeof(WarpStage) * (kMaxTPB / 32) <= 48 * 1024, "static shared memory of the camera stage");

// Lane 0 only: take the block's lock, at most 64 tries.
__device__ __forceinline__ bool bank_try_lock(int* lock) {
  for (int k = 0; k < 64; ++k) {
    if (atomicCAS(lock, 0, 1) == 0) {
      __threadfence_block();
      return true;
    }
    __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void bank_unlock(int* lock) {
  __threadfence_block();
  atomicExch(lock, 0);
}
// The whole warp: lane 0 tries the lock, every lane learns the outcome; the
// warp barrier orders lane 0's acquire before the other lanes' accesses.
__device__ __forceinline__ bool warp_lock(int* lock, int lane) {
  int got = 0;
  if (lane == 0) got = bank_try_lock(lock);
  got = __shfl_sync(kFull, got, 0);
  __syncwarp();
  return got != 0;
}
__device__ __forceinline__ void warp_unlock(int* lock, int lane) {
  __syncwarp();
  if (lane == 0) bank_unlock(lock);
  __syncwarp();
}
__device__ __forceinline__ int shared_load(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ void shared_store(int* p, int v) { *reinterpret_cast<volatile int*>(p) = v; }
// Lane 0's view of a bank counter, for every lane (a warp-uniform hint).
__device__ __forceinline__ int warp_peek(const int* p, int lane) {
  int v = 0;
  if (lane == 0) v = shared_load(p);
  return __shfl_sync(kFull, v, 0);
}

// Request loop: a parked warp that found work leaves the park count, unless
// the kernel is closing (lane 0; bounded number of tries).
__device__ __forceinline__ bool serve_unpark(unsigned long long* park) {
  for (int t = 0; t < 64; ++t) {
    const unsigned long long w = *reinterpret_cast<volatile unsigned long long*>(park);
    if (w >> 63) return false;
    if (atomicCAS(park, w, w - 1ull) == w) return true;
  }
  return false;
}

__device__ __forceinline__ unsigned nsmid() {
  unsigned n;
  asm("mov.u32 %0, %%nsmid;" : "=r"(n));
  return n;
}

// Zone-warp waits that ran out (TraceParams::zone_wait_ns), device-wide: a
// zone warp that has been without work for that long while other warps of
// its block still run closes its bank and leaves (the others then take their
// zone steps in place, with the same arithmetic) and counts itself here.
__device__ unsigned long long g_wait_timeouts;

static_assert(kHamKerrBL == MALBEC_FORM_HAMILTONIAN && kHamAdm == MALBEC_FORM_ADM, "form codes");

// (x, u) -> (x, p): p = g u, with g of eq. kerr or of the 3+1 quantities.
template <int kForm>
__device__ __forceinline__ void to_momenta(double M, double a, const double y[8], double p[4]) {
  if constexpr (kForm == kHamAdm) {
    Adm<double> m;
    adm_kerr<double>(make_bh<double>(M, a), y[1], y[2], m);
    adm_lower(m, y + 4, p);
  } else {
    lower_velocity(M, a, y, p);
  }
}

// (x, p) -> u = g^{-1} p, the inverse of to_momenta.
template <int kForm>
__device__ __forceinline__ void to_velocity(double M, double a, const double z[8], double u[4]) {
  if constexpr (kForm == kHamAdm) {
    Adm<double> m;
    adm_kerr<double>(make_bh<double>(M, a), z[1], z[2], m);
    adm_raise(m, z + 4, u);
  } else {
    raise_momentum(M, a, z, u);
  }
}

// Launch bounds: at most kMaxTPB threads per block, one block per SM
// guaranteed.  The kernel runs one to twelve warps per SM (see choose_shape),
// and the register budget is left to the compiler; without the
// minimum-blocks argument it gives every instantiation fewer registers (the
// FP32_MIXED camera kernel 146 instead of 190, and 1.9x slower: 20.5 against
// 10.8 ms per 1024^2 render; some request-loop instantiations were capped at
// 128 and spilled).  Two RK4 exceptions are held to 168 registers, so that three
// 128-thread blocks fit an SM (3 x 128 x 168 <= 65536): the FP32_MIXED
// job-table kernel with the block ray exchange, whose autotuned shape is
// three blocks per SM (with 176 registers it ran on two, and the 4096 uneven
// bundles took 32.7 s against 27.4 s), and the FP32_MIXED whole-image camera
// kernels, which are latency-bound with two warps per SM sub-partition (8 B
// of spills at 168; 1024^2 render 9.4-9.7 ms on three blocks per SM against
// 11.0 ms on two with 194 registers; at 128 registers, four blocks per SM:
// 13.8 ms).
template <bool kMixed, int kSrc, bool kBanks, int kMethod>
constexpr int trace_reg_cap() {
  return kMethod == MALBEC_METHOD_RK4 &&
                 ((kMixed && kBanks && kSrc == kSrcJobs) || (kMixed && !kBanks && kSrc == kSrcCamera))
             ? 168
             : 255;
}

template <bool kKerr, bool kMixed, int kSrc, int kSink, bool kBanks, int kForm, int kMethod>
__global__ void __launch_bounds__(kMaxTPB, 1) __maxnreg__((trace_reg_cap<kMixed, kSrc, kBanks, kMethod>()))
    trace_kernel(const TraceParams p) {
  static_assert(!kBanks || kMixed, "block banks exist for FP32_MIXED only");
  constexpr bool kHam = kForm != MALBEC_FORM_GEODESIC;
  static_assert(!kHam || kKerr, "the canonical forms use the Kerr Hamiltonian (a = 0 included)");
  constexpr bool kDopri = kMethod == MALBEC_METHOD_DOPRI5;
  static_assert(!kDopri || !kMixed || !kBanks, "FP32_MIXED Dormand-Prince: no block exchange");
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const float k6h = (float)(1.0 / 6.0), k6l = (float)(1.0 / 6.0 - (double)(float)(1.0 / 6.0));
  const float pole_f = (float)p.zone_pole;
  // Step rule and termination of the lane's ray: uniform, except for rays of
  // a job table, which carry their job's values.
  double M = p.M, dl = p.dl, dl_scale = p.dl_r_scale, r_esc = p.r_esc, eps_hor = p.eps_hor;
  double rtol = p.rtol, atol = p.atol;
  uint32_t cap = p.cap;
  // FP32-path constants: fixed step as a float pair, 1/6 as a float pair
  float h_fix, h6_fix_h, h6_fix_l, scale_f, r_esc_f;
  step_consts(dl, dl_scale, r_esc, h_fix, h6_fix_h, h6_fix_l, scale_f, r_esc_f);
  uint32_t job = 0;

  double y[8];
  float hi[8], lo[8];
  double lam = 0.0;
  uint32_t nst = 0;
  uint64_t id = 0;
  double a = p.a, r_cap = 0.0;
  // validity flag: the norm g(u,u) at the start and the largest departure
  // from it that the end state may show (MALBEC_FATE_DRIFTED)
  double n0 = 0.0, drift_lim = 0.0;
  float r_cap_f = 0.f, r_zone_f = 0.f, pole_lane = -1.f;
  // FP64 kernels: constant operands in per-thread registers (make_bh); the
  // FP32_MIXED kernels keep their register budget for the FP32 state
  const unsigned long long vz = kMixed ? 0ull : ((unsigned long long)threadIdx.x & p.lane_zero);
  BH<double> bh64 = make_bh<double>(M, p.a, vz);
  BH<float> bh32 = make_bh<float>(M, p.a);
  int zone_waited = 0;
  unsigned long long idle_since = 0ull, nap_since = 0ull;
  int claim_backoff = 0;
  bool active = false, drained = false, parked = false;
  // FP32 steps add their h to a float pair (TwoSum), flushed into the FP64
  // lambda after every 32nd step of the ray, before an FP64 step and at the
  // end (a fixed step only counts): no FP64 operation in the FP32 bulk step,
  // and the flush points depend on the ray's own steps alone.
  float lam_h = 0.f, lam_l = 0.f;
  uint32_t lam_fix = 0;
  // Dormand-Prince: the next step size, f(y) of the accepted state (the
  // first stage of the next attempt) and whether the last attempt failed
  double h_next = 0.0, k1d[8];
  bool after_reject = false;
  // FP32_MIXED Dormand-Prince: the next step size and k1 in FP32, the
  // tolerances in FP32
  float hn_f = 0.f, k1f[8];
  float rtol_f = (float)p.rtol, atol_f = (float)p.atol;  // per job from job tables
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    k1d[c] = 0.0;
    k1f[c] = 0.f;
    y[c] = 0.0;
    hi[c] = 0.f;
    lo[c] = 0.f;
  }
  auto flush_lam = [&]() {
    lam += ((double)lam_h + (double)lam_l) + (double)lam_fix * dl;
    lam_h = lam_l = 0.f;
    lam_fix = 0;
  };

  // Block banks (FP32_MIXED with at least two warps per block).
  __shared__ typename BanksFor<kBanks>::type banks;
  const int n_warps = (int)(blockDim.x >> 5);
  const bool use_banks = kBanks && n_warps >= 2;
  const int zone_warp_index = use_banks ? (int)((blockIdx.x / nsmid()) % (unsigned)n_warps) : -1;
  const bool zone_warp = (int)(threadIdx.x >> 5) == zone_warp_index;
  if constexpr (kBanks) {
    if (threadIdx.x == 0) {
      banks.n_zone = 0;
      banks.n_fp32 = 0;
      banks.lock = 0;
      banks.open = use_banks ? 1 : 0;
      banks.alive = n_warps - 1;
    }
    __syncthreads();
  }
  // Move this lane's ray into / out of bank slot s (FP32_MIXED only).
  auto save_ray = [&](RayBank& b, int s) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      b.hi[c][s] = hi[c];
      b.lo[c][s] = lo[c];
    }
    b.lam[s] = lam;
    b.M[s] = M;
    b.a[s] = a;
    b.dl[s] = dl;
    b.dls[s] = dl_scale;
    b.r_esc[s] = r_esc;
    b.r_cap[s] = r_cap;
    b.id[s] = id;
    b.job[s] = job;
    b.nst[s] = nst;
    b.cap[s] = cap;
    b.r_zone[s] = r_zone_f;
    b.pole[s] = pole_lane;
    b.lam_h[s] = lam_h;
    b.lam_l[s] = lam_l;
    b.lam_fix[s] = lam_fix;
    b.n0[s] = n0;
    b.drift_lim[s] = drift_lim;
    active = false;
  };
  auto load_ray = [&](const RayBank& b, int s) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      hi[c] = b.hi[c][s];
      lo[c] = b.lo[c][s];
    }
    lam = b.lam[s];
    M = b.M[s];
    a = b.a[s];
    dl = b.dl[s];
    dl_scale = b.dls[s];
    r_esc = b.r_esc[s];
    r_cap = b.r_cap[s];
    id = b.id[s];
    job = b.job[s];
    nst = b.nst[s];
    cap = b.cap[s];
    r_zone_f = b.r_zone[s];
    pole_lane = b.pole[s];
    step_consts(dl, dl_scale, r_esc, h_fix, h6_fix_h, h6_fix_l, scale_f, r_esc_f);
    bh64 = make_bh<double>(M, a);
    bh32 = make_bh<float>(M, a);
    r_cap_f = (float)r_cap;
    zone_waited = 0;
    lam_h = b.lam_h[s];
    lam_l = b.lam_l[s];
    lam_fix = b.lam_fix[s];
    n0 = b.n0[s];
    drift_lim = b.drift_lim[s];
    active = true;
  };
  auto zone_test = [&]() -> bool {
    return active && nst < cap && (hi[1] < r_zone_f || fabsf(__sinf(hi[2])) < pole_lane);
  };
  // A warp with no ray left asks to leave (banks in use).  The zone warp
  // leaves once its bank is empty and every other warp of the block has left
  // (it naps meanwhile, at most p.zone_wait_ns, then closes its bank and
  // counts the expiry); the others leave once the FP32 bank is empty.
  // Returns false to loop again.
  auto leave_block_banks = [&](auto& bk) -> bool {
    if (!warp_lock(&bk.lock, lane)) return false;
    int leave = 0;
    if (lane == 0) {
      if (zone_warp) {
        const int nz = shared_load(&bk.n_zone), alive = shared_load(&bk.alive);
        if (nz == 0) {
          const unsigned long long now = global_ns();
          if (nap_since == 0ull) nap_since = now;
          if (alive == 0 || now - nap_since > p.zone_wait_ns) {
            if (alive != 0) atomicAdd(&g_wait_timeouts, 1ull);
            shared_store(&bk.open, 0);
            leave = 1;
          }
        }
      } else if (shared_load(&bk.n_fp32) == 0) {
        shared_store(&bk.alive, shared_load(&bk.alive) - 1);
        leave = 1;
      }
    }
    leave = __shfl_sync(kFull, leave, 0);
    warp_unlock(&bk.lock, lane);
    if (!leave && zone_warp) __nanosleep(1000);
    return leave != 0;
  };

  // Quantities fixed at a ray's start: the norm at the start and the drift
  // limit of the validity flag, and (FP32_MIXED) the FP64-zone radius and
  // polar threshold, which differ between null rays and particles.
  auto start_consts = [&](const double ys[8], const double inv[4], double rp, double& n0_s, double& dlim_s,
                          float& rz_s, float& pole_s) {
    n0_s = inv[3];
    dlim_s = MALBEC_NORM_DRIFT_TOL * fmax(inv[0] * inv[0], fabs(inv[3]));
    if constexpr (kMixed) {
      const double cth = cos(ys[2]);
      const double gtt = 2.0 * M * ys[1] / fma(a * a, cth * cth, ys[1] * ys[1]) - 1.0;
      const bool is_null = fabs(inv[3]) <= 1e-6 * fabs(gtt) * ys[4] * ys[4];
      double rz = p.zone_horizon * rp;
      if (is_null) rz = fmax(rz, dev_r_photon_retro(M, a) + p.zone_photon * M);
      rz_s = (float)rz;
      pole_s = is_null ? -1.f : pole_f;
    }
  };

  // FP64 whole-image cameras: the warp's stage (see WarpStage).  The black
  // hole, the capture radius and the step rule are the same for every pixel.
  constexpr bool kStage = kSrc == kSrcCamera && kSink == kSinkCamera && !kMixed;
  __shared__ typename StageFor<kStage>::type stage;
  const int warp_in_block = (int)(threadIdx.x >> 5);
  double rp_cam = 0.0;
  int st_left = 0, st_pos = 0, e_n = 0;  // warp-uniform: staged starts left, next one; staged ends
  bool q_done = false, pend = false;      // queue exhausted; this lane's ray ended, not yet staged
  uint32_t end_fate = 0;
  if constexpr (kStage) {
    rp_cam = dev_r_plus(M, a);
    r_cap = (1.0 + eps_hor) * rp_cam;
  }
  // Lane l prepares the start of pixel pix in slot l.
  auto stage_start = [&](WarpStage& ws, unsigned long long pix) {
    double ys[8], inv[4];
    camera_state(p.cam, a, pix, ys);
    invariants64(M, a, ys, inv);
    double n0_s, dlim_s;
    float rz_s = 0.f, pole_s = -1.f;  // FP32_MIXED only
    start_consts(ys, inv, rp_cam, n0_s, dlim_s, rz_s, pole_s);
    if constexpr (kHam) {
      double pz[4];
      to_momenta<kForm>(M, a, ys, pz);
#pragma unroll
      for (int c = 0; c < 4; ++c) ys[4 + c] = pz[c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) ws.y0[c][lane] = ys[c];
    ws.n0[lane] = n0_s;
    ws.dlim0[lane] = dlim_s;
    ws.id0[lane] = pix;
  };
  // This lane's ended ray into end slot s (its state has not changed since
  // it ended: an idle lane is not stepped).
  auto stage_end = [&](WarpStage& ws, int s) {
#pragma unroll
    for (int c = 1; c < 8; ++c) ws.y1[c - 1][s] = y[c];
    ws.n1[s] = n0;
    ws.dlim1[s] = drift_lim;
    ws.id1[s] = id;
    ws.nst1[s] = nst;
    ws.fate1[s] = end_fate;
  };
  // The whole warp finishes the n staged ends: end invariants, validity flag,
  // the pixel's outputs.
  auto finish_ends = [&](WarpStage& ws, int n) {
    __syncwarp();
    if (lane < n) {
      double ye[8];
      ye[0] = 0.0;  // t enters neither the invariants nor the outputs
#pragma unroll
      for (int c = 1; c < 8; ++c) ye[c] = ws.y1[c - 1][lane];
      if constexpr (kHam) {
        double u[4];
        to_velocity<kForm>(M, a, ye, u);
#pragma unroll
        for (int c = 0; c < 4; ++c) ye[4 + c] = u[c];
      }
      double inv1[4];
      invariants64(M, a, ye, inv1);
      uint32_t f = ws.fate1[lane];
      if ((f == MALBEC_FATE_ESCAPED || f == MALBEC_FATE_CAPPED) && fabs(inv1[3] - ws.n1[lane]) > ws.dlim1[lane])
        f |= MALBEC_FATE_DRIFTED;
      const unsigned long long i = ws.id1[lane];
      p.fate_out[i] = (uint8_t)f;
      p.steps_out[i] = ws.nst1[lane];
      p.theta_out[i] = ye[2];
      p.phi_out[i] = ye[3];
    }
    __syncwarp();
  };

  while (true) {
    if constexpr (kStage) {
      // rays that ended in the last warp step go to the stage
      const unsigned pm = __ballot_sync(kFull, pend);
      if (pm != 0u) {
        WarpStage& ws = stage[warp_in_block];
        if (e_n + __popc(pm) > 32) {
          finish_ends(ws, e_n);
          e_n = 0;
        }
        if (pend) {
          stage_end(ws, e_n + __popc(pm & lt_mask));
          pend = false;
        }
        e_n += __popc(pm);
      }
    }
    unsigned act = __ballot_sync(kFull, active);
    if constexpr (kBanks) {
      if (use_banks) {
        if (zone_warp) {
          // ---- zone warp: take waiting zone rays into idle lanes, handing
          // FP32 rays to the FP32 bank to make room for them
          if (warp_peek(&banks.n_zone, lane) > 0 && warp_lock(&banks.lock, lane)) {
            const unsigned cand = __ballot_sync(kFull, active && !zone_test());
            int nz = 0, nf = 0, alive = 0;
            if (lane == 0) {
              nz = shared_load(&banks.n_zone);
              nf = shared_load(&banks.n_fp32);
              alive = shared_load(&banks.alive);
            }
            nz = __shfl_sync(kFull, nz, 0);
            nf = __shfl_sync(kFull, nf, 0);
            alive = __shfl_sync(kFull, alive, 0);
            const int n_idle = 32 - __popc(act);
            unsigned evict = 0u;
            if (nz > n_idle && alive > 0) {
              int k = min(nz - n_idle, __popc(cand));
              k = min(k, kBankSlots - nf);
              const unsigned rank = __popc(cand & lt_mask);
              evict = __ballot_sync(kFull, ((cand >> lane) & 1u) && (int)rank < k);
              if ((evict >> lane) & 1u) save_ray(banks.fp32, nf + (int)rank);
              nf += __popc(evict);
            }
            const unsigned free_lanes = ~act | evict;
            const int take = min(nz, __popc(free_lanes));
            const unsigned frank = __popc(free_lanes & lt_mask);
            if (((free_lanes >> lane) & 1u) && (int)frank < take) load_ray(banks.zone, nz - 1 - (int)frank);
            if (lane == 0) {
              shared_store(&banks.n_zone, nz - take);
              shared_store(&banks.n_fp32, nf);
            }
            warp_unlock(&banks.lock, lane);
            act = __ballot_sync(kFull, active);
          }
        } else if (act != kFull && warp_peek(&banks.n_fp32, lane) > 0 && warp_lock(&banks.lock, lane)) {
          // ---- other warps: rays the zone warp handed back go first
          int nf = 0;
          if (lane == 0) nf = shared_load(&banks.n_fp32);
          nf = __shfl_sync(kFull, nf, 0);
          const unsigned free_lanes = ~act;
          const int take = min(nf, __popc(free_lanes));
          const unsigned frank = __popc(free_lanes & lt_mask);
          if (((free_lanes >> lane) & 1u) && (int)frank < take) load_ray(banks.fp32, nf - 1 - (int)frank);
          if (lane == 0) shared_store(&banks.n_fp32, nf - take);
          warp_unlock(&banks.lock, lane);
          act = __ballot_sync(kFull, active);
        }
      }
    }
    const int idle = 32 - __popc(act);
    if (kSrc == kSrcServe && claim_backoff > 0) --claim_backoff;
    if (!drained && idle > 0 && (idle >= p.refill_min || act == 0) && (act == 0 || claim_backoff == 0)) {
      bool got = false;
      if constexpr (kStage) {
        // ---- idle lanes take staged starts; an empty stage is refilled with
        // the next 32 pixels of the queue (near the end of the queue, with
        // as many as there are idle lanes, so that no warp holds back rays
        // that other warps could take)
        WarpStage& ws = stage[warp_in_block];
        unsigned need = ~act;
        while (need != 0u) {
          if (st_left == 0) {
            if (q_done) break;
            __syncwarp();  // every slot has been read before it is rewritten
            unsigned long long base = 0;
            int want = 32;
            if (lane == 0) {
              const unsigned long long reserve = 2ull * gridDim.x * blockDim.x;
              const unsigned long long h = *reinterpret_cast<volatile unsigned long long*>(p.head);
              if (h >= p.n || p.n - h <= reserve) want = __popc(need);
              base = atomicAdd(p.head, (unsigned long long)want);
            }
            base = __shfl_sync(kFull, base, 0);
            want = __shfl_sync(kFull, want, 0);
            if (base + (unsigned long long)want >= p.n) q_done = true;
            const int k = base < p.n ? (int)min((unsigned long long)want, p.n - base) : 0;
            if (lane < k) stage_start(ws, camera_claim_pixel(p.cam, base + (unsigned long long)lane));
            __syncwarp();
            st_left = k;
            st_pos = 0;
            if (k == 0) break;
          }
          const int take = min(__popc(need), st_left);
          const unsigned rank = __popc(need & lt_mask);
          const bool mine = ((need >> lane) & 1u) && (int)rank < take;
          if (mine) {
            const int s = st_pos + (int)rank;
#pragma unroll
            for (int c = 0; c < 8; ++c) y[c] = ws.y0[c][s];
            n0 = ws.n0[s];
            drift_lim = ws.dlim0[s];
            id = ws.id0[s];
            got = true;
          }
          need &= ~__ballot_sync(kFull, mine);
          st_pos += take;
          st_left -= take;
        }
        drained = q_done && st_left == 0;
      } else if (kSrc == kSrcStates || kSrc == kSrcCamera) {
        // ---- hand the next `idle` rays of the queue to the idle lanes
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(p.head, (unsigned long long)idle);
        base = __shfl_sync(kFull, base, 0);
        if (base + (unsigned long long)idle >= p.n) drained = true;
        const unsigned long long my = base + __popc(~act & lt_mask);
        if (!active && my < p.n) {
          id = kSrc == kSrcCamera ? camera_claim_pixel(p.cam, my) : my;
          got = true;
        }
      } else if (kSrc == kSrcServe) {
        // ---- claim rays from the active jobs, in the order the host
        // publishes (smallest first): the warp reads 32 entries of the list
        // at a time and lane 0 claims from the first job that has rays left,
        // until every idle lane has a ray or no listed job has rays left; no
        // new claims once the host asked to stop.  A job whose last rays went
        // to another warp meanwhile is seen exhausted on the next look.
        unsigned need = ~act;
        uint32_t na = 0, stop = 0;
        if (lane == 0) {
          na = *p.active_count;
          stop = *p.stop_flag;
        }
        na = __shfl_sync(kFull, na, 0);
        stop = __shfl_sync(kFull, stop, 0);
        if (na > p.max_active) na = p.max_active;
        uint32_t i0 = 0;
        while (need != 0u && stop == 0u && i0 < na) {
          const uint32_t i = i0 + (uint32_t)lane;
          uint32_t s = 0;
          unsigned long long ns = 0;
          bool avail = false;
          if (i < na) {
            const uint64_t jid = p.active_ids[i];
            if (jid != 0) {
              s = (uint32_t)(jid % p.n_jobs);
              if (__ldcg(reinterpret_cast<const unsigned long long*>(&p.jobs[s].job_id)) == jid) {
                ns = __ldcg(reinterpret_cast<const unsigned long long*>(&p.jobs[s].n));
                avail = *reinterpret_cast<volatile unsigned long long*>(&p.job_ctr[s].next) < ns;
              }
            }
          }
          const unsigned m = __ballot_sync(kFull, avail);
          if (m == 0u) {
            i0 += 32u;
            continue;
          }
          if (parked) {
            int ok = 0;
            if (lane == 0) ok = serve_unpark(p.park);
            if (__shfl_sync(kFull, ok, 0) == 0) break;  // closing: claim nothing
            parked = false;
          }
          const int first = __ffs(m) - 1;
          s = __shfl_sync(kFull, s, first);
          ns = __shfl_sync(kFull, ns, first);
          const int cnt = __popc(need);
          unsigned long long b = 0;
          if (lane == 0) b = atomicAdd(&p.job_ctr[s].next, (unsigned long long)cnt);
          b = __shfl_sync(kFull, b, 0);
          if (b >= ns) continue;
          const unsigned long long n_take = ns - b < (unsigned long long)cnt ? ns - b : (unsigned long long)cnt;
          const bool mine = (need >> lane) & 1u;
          const unsigned rank = __popc(need & lt_mask);
          const bool take_it = mine && rank < n_take;
          if (take_it) {
            job = s;
            id = b + rank;
            got = true;
          }
          need &= ~__ballot_sync(kFull, take_it);
        }
      } else {
        // ---- claim rays job by job, costliest jobs first, until every idle
        // lane has one or the table is exhausted
        unsigned need = ~act;
        while (need != 0u) {
          const int cnt = __popc(need);
          unsigned cur = 0;
          unsigned long long base = 0;
          if (lane == 0) {
            cur = *reinterpret_cast<volatile unsigned*>(p.job_cursor);
            if (cur < p.n_jobs) base = atomicAdd(&p.job_ctr[p.job_order[cur]].next, (unsigned long long)cnt);
          }
          cur = __shfl_sync(kFull, cur, 0);
          base = __shfl_sync(kFull, base, 0);
          if (cur >= p.n_jobs) {
            drained = true;
            break;
          }
          const uint32_t jidx = p.job_order[cur];
          const unsigned long long nj = p.jobs[jidx].n;
          const unsigned long long avail = base < nj ? (nj - base < (unsigned long long)cnt ? nj - base : cnt) : 0ull;
          if (avail < (unsigned long long)cnt && lane == 0) atomicCAS(p.job_cursor, cur, cur + 1u);
          const bool mine = (need >> lane) & 1u;
          const unsigned rank = __popc(need & lt_mask);
          const bool take_it = mine && rank < avail;
          if (take_it) {
            job = jidx;
            id = base + rank;
            got = true;
          }
          need &= ~__ballot_sync(kFull, take_it);
        }
      }
      if (kSrc == kSrcServe) {
        // no ray for any lane of this warp: nap.  After idle_ns of idleness
        // the warp parks; the kernel leaves once every warp is parked (all
        // at once: the first to see it closes, and a parked warp that finds
        // work unparks before it claims), or when the host asks to stop.
        // Lane 0 decides; every wait is a bounded nap of the loop.
        if (act == 0 && __ballot_sync(kFull, got) == 0u) {
          bool quit = false;
          if (lane == 0) {
            const unsigned long long now = global_ns();
            if (idle_since == 0ull) idle_since = now;
            volatile unsigned long long* pk = p.park;
            if ((*pk >> 63) != 0ull || *p.stop_flag != 0u) {
              quit = true;
            } else {
              if (!parked && now - idle_since > p.idle_ns) {
                atomicAdd(p.park, 1ull);
                parked = true;
              }
              if (parked) {
                const unsigned long long w = *pk;
                const unsigned long long total = (unsigned long long)gridDim.x * (blockDim.x >> 5);
                if ((w >> 63) != 0ull)
                  quit = true;
                else if ((w & 0xffffffffull) == total && atomicCAS(p.park, w, w | (1ull << 63)) == w)
                  quit = true;
              }
            }
          }
          parked = __shfl_sync(kFull, parked, 0);
          if (__shfl_sync(kFull, quit, 0)) {
            if constexpr (kBanks) {
              if (!use_banks || leave_block_banks(banks)) break;
            } else {
              break;
            }
          }
          __nanosleep(2000);
          continue;
        }
        idle_since = 0ull;
        // busy lanes but nothing to claim: look again after 32 warp steps
        if (__ballot_sync(kFull, got) == 0u) claim_backoff = 32;
      }
      if (got) {
        active = true;
        if (kSrc == kSrcJobs || kSrc == kSrcServe) {
          const JobDesc J = load_job(&p.jobs[job]);
          M = J.M;
          a = J.a;
          dl = J.dl;
          dl_scale = J.dl_r_scale;
          r_esc = J.r_esc;
          eps_hor = J.eps_hor;
          cap = J.cap;
          rtol = J.rtol;
          atol = J.atol;
          if constexpr (kMixed && kDopri) {
            rtol_f = (float)rtol;
            atol_f = (float)atol;
          }
          step_consts(dl, dl_scale, r_esc, h_fix, h6_fix_h, h6_fix_l, scale_f, r_esc_f);
          if (J.kind == MALBEC_BUNDLE_CAMERA) {
            camera_state(J.cam, a, id, y);
          } else if (J.kind == MALBEC_BUNDLE_BOUND) {
            double a_s;
            bound_sample(M, a, 1, J.seed, id, y, &a_s);
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) y[c] = J.ics[(size_t)c * J.n + id];
          }
        } else if (kSrc == kSrcStates) {
#pragma unroll
          for (int c = 0; c < 8; ++c) y[c] = p.ics[(size_t)c * p.n + id];
          if (p.a_per_ray) a = p.a_per_ray[id];
        } else if constexpr (!kStage) {
          camera_state(p.cam, a, id, y);
        }
        lam = 0.0;
        lam_h = lam_l = 0.f;
        lam_fix = 0;
        nst = 0;
        zone_waited = 0;
        if constexpr (!kStage) {
          // (staged camera rays: state (x, u) or (x, p), n0 and drift_lim
          // came from the stage; black hole and capture radius are fixed)
          bh64 = make_bh<double>(M, a, vz);
          if (kMixed) bh32 = make_bh<float>(M, a);
          const double rp = dev_r_plus(M, a);
          r_cap = (1.0 + eps_hor) * rp;
          const bool from_jobs = kSrc == kSrcJobs || kSrc == kSrcServe;
          const JobDesc* Jp = from_jobs ? &p.jobs[job] : nullptr;
          const bool camera_ray =
              kSink == kSinkCamera ||
              (from_jobs && __ldcg(reinterpret_cast<const int*>(&Jp->kind)) == MALBEC_BUNDLE_CAMERA);
          {
            double inv[4];
            invariants64(M, a, y, inv);
            start_consts(y, inv, rp, n0, drift_lim, r_zone_f, pole_lane);
            if (!camera_ray) {
              double* inv0 = from_jobs ? reinterpret_cast<double*>(
                                             __ldcg(reinterpret_cast<const unsigned long long*>(&Jp->inv0_out)))
                                       : p.inv0_out;
              const uint64_t nn = from_jobs ? __ldcg(reinterpret_cast<const unsigned long long*>(&Jp->n)) : p.n;
#pragma unroll
              for (int c = 0; c < 4; ++c) inv0[(size_t)c * nn + id] = inv[c];
            }
            if (kMixed) {
              r_cap_f = (float)r_cap;
              split_pair(y, hi, lo);
            }
          }
          if (kSink == kSinkStrided) store_sample<kMixed>(p, a, id, 0, y, hi);
          if constexpr (kHam) {
            // canonical form: integrate (x, p) with p = g u
            double pz[4];
            to_momenta<kForm>(M, a, y, pz);
#pragma unroll
            for (int c = 0; c < 4; ++c) y[4 + c] = pz[c];
            if constexpr (kMixed) split_pair(y, hi, lo);
          }
        }
        if constexpr (kDopri) {
          // first trial step; k1 = f(y) for the first attempt
          h_next = dl > 0.0 ? dl : dl_scale * y[1];
          after_reject = false;
          if constexpr (kHam) {
            double f[6];
            ham_rhs<kForm, double>(bh64, y[1], y[2], y[4], y[5], y[6], y[7], f);
#pragma unroll
            for (int c = 0; c < 4; ++c) k1d[c] = f[c];
            k1d[4] = 0.0;
            k1d[5] = f[4];
            k1d[6] = f[5];
            k1d[7] = 0.0;
          } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) k1d[c] = y[4 + c];
            accel<kKerr, double>(bh64, y[1], y[2], y[4], y[5], y[6], y[7], k1d + 4);
          }
          if constexpr (kMixed) {
            hn_f = (float)h_next;
#pragma unroll
            for (int c = 0; c < 8; ++c) k1f[c] = (float)k1d[c];
          }
        }
      }
      continue;
    }
    if (act == 0) {  // queue drained and no lane busy
      if constexpr (kBanks) {
        if (!use_banks || leave_block_banks(banks)) break;
        continue;
      } else {
        if constexpr (kStage) finish_ends(stage[warp_in_block], e_n);
        break;
      }
    }
    if (zone_warp) nap_since = 0ull;
    // FP32_MIXED: one warp step is either an FP64-zone step (for every lane
    // that wants one) or an FP32 step (for the others), never both.  FP64
    // steps are deferred until zone_batch lanes want one, no lane wants an
    // FP32 step, a waiting lane has sat out zone_wait warp steps, or (queue
    // drained) zone rays are a quarter of the live rays.  Only the timing of
    // a ray's steps changes, never their arithmetic.
    bool in_zone = false, take = true;
    if constexpr (kMixed) {
      in_zone = zone_test();
      unsigned m64 = __ballot_sync(kFull, in_zone);
      if constexpr (kBanks) {
        // too few zone rays here for an FP64 step: hand them to the zone warp
        if (use_banks && !zone_warp && m64 != 0u && __popc(m64) < p.zone_batch && warp_peek(&banks.open, lane) != 0 &&
            warp_peek(&banks.n_zone, lane) < kBankSlots && warp_lock(&banks.lock, lane)) {
          int nz = 0, open = 0;
          if (lane == 0) {
            nz = shared_load(&banks.n_zone);
            open = shared_load(&banks.open);
          }
          nz = __shfl_sync(kFull, nz, 0);
          open = __shfl_sync(kFull, open, 0);
          const int k = open ? min(__popc(m64), kBankSlots - nz) : 0;
          const unsigned rank = __popc(m64 & lt_mask);
          if (in_zone && (int)rank < k) {
            save_ray(banks.zone, nz + (int)rank);
            in_zone = false;
          }
          if (lane == 0) shared_store(&banks.n_zone, nz + k);
          warp_unlock(&banks.lock, lane);
          m64 = __ballot_sync(kFull, in_zone);
        }
      }
      const bool want32 = active && nst < cap && !in_zone;
      const unsigned m32 = __ballot_sync(kFull, want32);
      const unsigned urgent = __ballot_sync(kFull, in_zone && zone_waited >= p.zone_wait);
      // once this warp's queue is drained no new ray will join a batch:
      // step the zone rays when they are a quarter of the warp's live rays
      const bool do64 = m32 == 0 || urgent != 0 || __popc(m64) >= p.zone_batch ||
                        (drained && 4 * __popc(m64) >= __popc(m64 | m32));
      take = do64 ? in_zone : want32;
      if (in_zone) zone_waited = do64 ? 0 : zone_waited + 1;
    }
    if (!active) continue;
    if (kMixed && nst < cap && !take) continue;

    int fate = 0;
    if (nst < cap) {
      // ---- one RK4 step
      bool captured, escaped, finite;
      if constexpr (kDopri && kMixed) {
        // ---- one FP32_MIXED Dormand-Prince attempt: in FP64 in the zone (on
        // y = hi + lo, k1 taken from FP32), else in FP32 on (hi, lo); the same
        // tests and step rule as in FP64, in the attempt's precision
        float hf = hn_f;
        if (scale_f > 0.f) hf = fminf(hf, scale_f * hi[1]);
        bool accept;
        if (in_zone) {
          double yd[8], k1l[8], y5[8], e[8], k7[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            yd[c] = (double)hi[c] + (double)lo[c];
            k1l[c] = (double)k1f[c];
          }
          const double h = (double)hf;
          const double rmin = dopri5_attempt_call<kKerr, kForm>(bh64, h, yd, k1l, y5, e, k7);
          captured = (y5[1] <= r_cap) | (rmin <= r_cap);
          finite = finite8(y5);
          escaped = false;
          accept = captured || !finite;
          if (!accept) {
            const double err = dopri5_norm(bh64, yd, y5, e, rtol, atol);
            accept = err <= 1.0;
            hn_f = (float)(h * dopri5_factor(err, accept, after_reject));
            after_reject = !accept;
            if (accept) {
#pragma unroll
              for (int c = 0; c < 8; ++c) k1f[c] = (float)k7[c];
              escaped = y5[1] >= r_esc;
            }
          }
          if (accept) {
            split_pair(y5, hi, lo);
            flush_lam();
            lam += h;
          }
        } else {
          float dx[8], dxe[8], e[8], k7[8], y5h[8];
          const float rmin = dopri5_attempt_mixed<kKerr, kForm>(bh32, hf, hi, lo, k1f, dx, dxe, e, k7);
#pragma unroll
          for (int c = 0; c < 8; ++c) y5h[c] = hi[c] + dx[c];
          captured = (y5h[1] <= r_cap_f) | (rmin <= r_cap_f);
          finite = finite8f(y5h);
          escaped = false;
          accept = captured || !finite;
          if (!accept) {
            const float err = dopri5_norm_f(hi, y5h, e, rtol_f, atol_f);
            accept = err <= 1.f;
            hn_f = hf * dopri5_factor_f(err, accept, after_reject);
            after_reject = !accept;
            if (accept) {
#pragma unroll
              for (int c = 0; c < 8; ++c) k1f[c] = k7[c];
              escaped = y5h[1] >= r_esc_f;
            }
          }
          if (accept) {
#pragma unroll
            for (int c = 0; c < 8; ++c) comp_add(hi[c], lo[c], dx[c], dxe[c]);
            float ls, le;
            two_sum(lam_h, hf, ls, le);
            lam_h = ls;
            lam_l += le;
            if ((nst & 31u) == 31u) flush_lam();
          }
        }
      } else if constexpr (kDopri) {
        // ---- one Dormand-Prince attempt: capture and non-finite on the
        // attempted state, acceptance by the error norm, escape on accepted
        // states; the step size adapts after every attempt
        if (dl_scale > 0.0) h_next = fmin(h_next, dl_scale * y[1]);
        const double h = h_next;
        double y5[8], e[8], k7[8];
        const double rmin = dopri5_attempt<kKerr, kForm>(bh64, h, y, k1d, y5, e, k7);
        captured = (y5[1] <= r_cap) | (rmin <= r_cap);
        finite = finite8(y5);
        escaped = false;
        bool accept = captured || !finite;
        if (!accept) {
          const double err = dopri5_norm(bh64, y, y5, e, rtol, atol);
          accept = err <= 1.0;
          h_next = h * dopri5_factor(err, accept, after_reject);
          after_reject = !accept;
          if (accept) {
#pragma unroll
            for (int c = 0; c < 8; ++c) k1d[c] = k7[c];
            escaped = y5[1] >= r_esc;
          }
        }
        if (accept) {
#pragma unroll
          for (int c = 0; c < 8; ++c) y[c] = y5[c];
          lam += h;
        }
      } else if (!kMixed) {
        const double h = dl_scale > 0.0 ? vmul(bh64, vreg(dl_scale, vz), y[1]) : dl;
        double rmin;
        if constexpr (kHam)
          rmin = rk4_step_ham<double, false, kForm>(bh64, h, y);
        else
          rmin = rk4_step<kKerr, double>(bh64, h, y);
        lam = vadd(bh64, lam, h);
        // the radius tests on the integer pipe (radius_key)
        const long long k1 = radius_key(y[1]);
        captured = key_le(k1, r_cap) | key_le(radius_key(rmin), r_cap);
        escaped = key_ge(k1, r_esc);
        finite = finite8(y);
      } else if (in_zone) {
        // FP64 zone (horizon, photon orbits, polar axis)
#pragma unroll
        for (int c = 0; c < 8; ++c) y[c] = (double)hi[c] + (double)lo[c];
        const double h = dl_scale > 0.0 ? dl_scale * y[1] : dl;
        double rmin;
        if constexpr (kHam)
          rmin = rk4_step_ham<double, true, kForm>(bh64, h, y);
        else
          rmin = rk4_step<kKerr, double, true>(bh64, h, y);
        flush_lam();
        lam += h;
        split_pair(y, hi, lo);
        const long long k1 = radius_key(y[1]);
        captured = key_le(k1, r_cap) | key_le(radius_key(rmin), r_cap);
        escaped = key_ge(k1, r_esc);
        finite = finite8(y);
      } else {
        float hf, h6h, h6l;
        if (scale_f > 0.f) {
          hf = scale_f * hi[1];
          h6h = hf * k6h;
          h6l = fmaf(hf, k6l, fmaf(hf, k6h, -h6h));
          float s, e;
          two_sum(lam_h, hf, s, e);
          lam_h = s;
          lam_l += e;
        } else {
          hf = h_fix;
          h6h = h6_fix_h;
          h6l = h6_fix_l;
          ++lam_fix;
        }
        if ((nst & 31u) == 31u) flush_lam();
        float rmin;
        if constexpr (kHam)
          rmin = rk4_step_mixed_ham<kForm>(bh32, hf, h6h, h6l, hi, lo);
        else
          rmin = rk4_step_mixed<kKerr>(bh32, hf, h6h, h6l, hi, lo);
        captured = (hi[1] <= r_cap_f) | (rmin <= r_cap_f);
        escaped = hi[1] >= r_esc_f;
        // a non-finite lo word comes with a non-finite hi word (lo is the
        // rounding error of hi's own sum), so the hi words decide
        finite = finite8f(hi);
      }
      ++nst;
      if (kSink == kSinkStrided && (nst % p.stride) == 0) {
        if (kHam && !p.traj_cartesian) {
          // canonical forms: the sample is (x, u), u = g^{-1} p
          double yz[8], yu[8];
          float hu[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) yz[c] = kMixed ? (double)hi[c] + (double)lo[c] : y[c];
#pragma unroll
          for (int c = 0; c < 4; ++c) yu[c] = yz[c];
          to_velocity<kForm>(M, a, yz, yu + 4);
#pragma unroll
          for (int c = 0; c < 8; ++c) hu[c] = (float)yu[c];
          store_sample<kMixed>(p, a, id, nst / p.stride, yu, hu);
        } else {
          store_sample<kMixed>(p, a, id, nst / p.stride, y, hi);
        }
      }
      // ---- termination tests, in the documented order
      if (captured)
        fate = MALBEC_FATE_CAPTURED;
      else if (!finite)
        fate = MALBEC_FATE_NONFINITE;
      else if (escaped)
        fate = MALBEC_FATE_ESCAPED;
      else if (nst >= cap)
        fate = MALBEC_FATE_CAPPED;
    } else {
      fate = MALBEC_FATE_CAPPED;  // n_steps_cap == 0
    }

    if (fate != 0) {
      if constexpr (kStage) {
        // staged at the top of the next warp step, finished with others
        pend = true;
        end_fate = (uint32_t)fate;
      } else if constexpr (kMixed && kSink == kSinkCamera) {
        // FP32_MIXED camera pixel: the validity flag from the norm of the
        // FP32 state in FP32 arithmetic (no FP64 work for one lane at a time:
        // its error, ~1e-6 of the largest term, is far inside the flag's
        // 1e-3 tolerance)
        const float nrm = state_norm_f<kHam>((float)M, (float)a, hi);
        if ((fate == MALBEC_FATE_ESCAPED || fate == MALBEC_FATE_CAPPED) && fabs((double)nrm - n0) > drift_lim)
          fate |= MALBEC_FATE_DRIFTED;
        p.fate_out[id] = (uint8_t)fate;
        p.steps_out[id] = nst;
        p.theta_out[id] = (double)hi[2] + (double)lo[2];
        p.phi_out[id] = (double)hi[3] + (double)lo[3];
      } else {
        if (kMixed) {
          flush_lam();
#pragma unroll
          for (int c = 0; c < 8; ++c) y[c] = (double)hi[c] + (double)lo[c];
        }
        if constexpr (kHam) {
          // back to (x, u) for the outputs and the invariants
          double u[4];
          to_velocity<kForm>(M, a, y, u);
#pragma unroll
          for (int c = 0; c < 4; ++c) y[4 + c] = u[c];
        }
        // the end invariants (FP64) and the validity flag
        double inv1[4];
        invariants64(M, a, y, inv1);
        if ((fate == MALBEC_FATE_ESCAPED || fate == MALBEC_FATE_CAPPED) && fabs(inv1[3] - n0) > drift_lim)
          fate |= MALBEC_FATE_DRIFTED;
        if (kSink == kSinkJobs) {
          const JobDesc J = load_job(&p.jobs[job]);
          if (J.kind == MALBEC_BUNDLE_CAMERA) {
            J.fate_out[id] = (uint8_t)fate;
            J.steps_out[id] = nst;
            J.theta_out[id] = y[2];
            J.phi_out[id] = y[3];
          } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) J.y_out[(size_t)c * J.n + id] = y[c];
            J.lambda_out[id] = lam;
            J.steps_out[id] = nst;
            J.fate_out[id] = (uint8_t)fate;
#pragma unroll
            for (int c = 0; c < 4; ++c) J.inv1_out[(size_t)c * J.n + id] = inv1[c];
          }
          // this ray's outputs are visible device-wide before it is counted
          __threadfence();
          const unsigned long long finished = atomicAdd(&p.job_ctr[job].done, 1ull) + 1ull;
          if (kSrc == kSrcServe && finished == J.n) {
            // last ray of the job: every output is visible, tell the host
            __threadfence_system();
            p.done_flags[job] = J.job_id;
          }
        } else if (kSink == kSinkCamera) {
          p.fate_out[id] = (uint8_t)fate;
          p.steps_out[id] = nst;
          p.theta_out[id] = y[2];
          p.phi_out[id] = y[3];
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) p.y_out[(size_t)c * p.n + id] = y[c];
          p.lambda_out[id] = lam;
          p.steps_out[id] = nst;
          p.fate_out[id] = (uint8_t)fate;
#pragma unroll
          for (int c = 0; c < 4; ++c) p.inv1_out[(size_t)c * p.n + id] = inv1[c];
          if (kSink == kSinkStrided) store_nan_samples<kMixed>(p, id, (uint64_t)nst / p.stride + 1);
        }
      }
      active = false;
    }
  }
}

template <bool kKerr, bool kMixed, int kSrc, int kSink, bool kBanks, int kForm = MALBEC_FORM_GEODESIC,
          int kMethod = MALBEC_METHOD_RK4>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&trace_kernel<kKerr, kMixed, kSrc, kSink, kBanks, kForm, kMethod>);
}

// The kernel for a launch; FP32_MIXED kernels come with and without the
// block ray exchange (two instantiations, so that the one without carries
// none of its code).
}  // namespace
}  // namespace malbec

// geodesic.cuh -- device-side geodesic right-hand sides, RK4 steps and
// conserved quantities for the Schwarzschild and Kerr metrics in
// Boyer-Lindquist coordinates (Quiroga, arXiv:1803.08320, Sec. 2 eq. kerr,
// Sec. 4 for a = 0).
//
// The acceleration du^mu/dl = -Gamma^mu_ab u^a u^b is evaluated per metric in
// closed form.  Kerr uses Gamma^mu_ab u^a u^b = g^{mu nu} W_nu with the
// first-kind contraction W_nu = Gamma_{nu ab} u^a u^b
//   = (d_a g_{nu b}) u^a u^b - 1/2 (d_nu g_ab) u^a u^b,
// which only needs the five metric components, their r- and theta-
// derivatives along u (the metric depends on r and theta alone) and the
// closed-form inverse of the (t, phi) block (det = -Delta sin^2); written
// through q = 2Mr/rho^2 and v = u^t - a sin^2 u^phi, the terms of the (t, phi)
// block collapse (see accel_kerr).  It is the same bilinear form as the twenty
// second-kind symbols of BL Kerr, with far fewer operations.  Schwarzschild
// uses its nine non-zero second-kind symbols
// directly.  One reciprocal per evaluation: 1/rho^2, 1/Delta and 1/sin^2 are
// products of 1/(rho^2 Delta sin^2).  In FP64 one sincos per RK4 step: the
// later stage angles take the angle-addition formulas (stage_trig).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace malbec {


// 1/x.  FP64: the hardware estimate (PTX rcp.approx.ftz.f64) refined by one
// step of the cubically convergent iteration y <- y (1 + e + e^2), e = 1 - x y
// (Newton's iteration for 1/x with the next term of the series 1/(1 - e)
// kept): the estimate's relative error e0 becomes O(e0^3) plus rounding.
// FP32: the estimate (rcp.approx.ftz.f32, within 1 ulp) refined by one
// Newton step y <- y + y (1 - x y), three instructions in place of the IEEE
// division's sequence (the 1024^2 FP32_MIXED camera: the same image, 5%
// faster).  Arguments here are positive and normal (products of rho^2,
// Delta, sin^2, far from the subnormal range).
// `one` is 1 (FP64: in a per-thread register, see vmul).
template <typename T>
__device__ __forceinline__ T recip(T x, T one);
template <>
__device__ __forceinline__ double recip<double>(double x, double one) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, one);
  return fma(y, fma(e, e, e), y);
}
template <>
__device__ __forceinline__ float recip<float>(float x, float) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return fmaf(y, fmaf(-x, y, 1.0f), y);
}
template <typename T>
__device__ __forceinline__ T recip(T x) {
  return recip<T>(x, T(1));
}

// ---------------------------------------------------------------------------
// FP64 operand forms.  On this part the FP64 unit takes an FMA whose operands
// are all per-thread registers (or two constant-bank operands) at its full
// rate, one warp instruction per ~64 cycles, but a DMUL, a DADD, or an FMA
// with an operand in a uniform register or mixed with one constant-bank
// operand takes ~18% longer (measured on GB300 with independent chains: 39.0
// against 33.0 ns per warp instruction; dependent chains run at the full rate
// too).  So the FP64 right-hand sides write a product as fma(x, y, -0) and a
// sum as fma(x, 1, y) -- exactly the IEEE product and sum, signed zeros, NaN
// and infinities included -- with -0, 1, the black-hole constants and the
// series coefficients held in per-thread registers: vreg(v, vz) is v with vz
// OR-ed into its bits, vz = threadIdx.x & (a launch parameter that is always
// 0), which the compiler can neither fold nor prove warp-uniform.  FP32: the
// plain operations.
__device__ __forceinline__ double vreg(double x, unsigned long long vz) {
  return __longlong_as_double(__double_as_longlong(x) | (long long)vz);
}

template <typename T>
struct BH {
  T M, a, a2, twoM, two_a2;
  T nz, one, two, half;  // -0, 1, 2, 1/2
  T k[10];               // k[n - 3] = 1/n!, n = 3..12 (the stage-angle series; k[0] = 1/6 also for h/6)
};

// vz = 0: the constants are whatever the compiler makes of them (any kernel
// may use that); per-thread registers when vz is the per-thread zero above.
template <typename T>
__device__ __forceinline__ BH<T> make_bh(double M, double a, unsigned long long vz = 0ull) {
  BH<T> b;
  double v[9] = {M, a, a * a, 2.0 * M, 2.0 * a * a, -0.0, 1.0, 2.0, 0.5};
  double f = 1.0;
  double k[10];
#pragma unroll
  for (int n = 1; n <= 12; ++n) {
    f *= (double)n;
    if (n >= 3) k[n - 3] = 1.0 / f;
  }
  if (sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = vreg(v[i], vz);
#pragma unroll
    for (int i = 0; i < 10; ++i) k[i] = vreg(k[i], vz);
  }
  b.M = T(v[0]);
  b.a = T(v[1]);
  b.a2 = T(v[2]);
  b.twoM = T(v[3]);
  b.two_a2 = T(v[4]);
  b.nz = T(v[5]);
  b.one = T(v[6]);
  b.two = T(v[7]);
  b.half = T(v[8]);
#pragma unroll
  for (int i = 0; i < 10; ++i) b.k[i] = T(k[i]);
  return b;
}

// x y, x + y, x - y in the full-rate operand form (FP64) or plainly (FP32).
template <typename T>
__device__ __forceinline__ T vmul(const BH<T>& b, T x, T y) {
  if constexpr (sizeof(T) == 8)
    return fma(x, y, b.nz);
  else
    return x * y;
}
template <typename T>
__device__ __forceinline__ T vadd(const BH<T>& b, T x, T y) {
  if constexpr (sizeof(T) == 8)
    return fma(x, b.one, y);
  else
    return x + y;
}
template <typename T>
__device__ __forceinline__ T vsub(const BH<T>& b, T x, T y) {
  if constexpr (sizeof(T) == 8)
    return fma(x, b.one, -y);
  else
    return x - y;
}

// sin and cos of an angle in FP64 on the FMA unit alone (the RK4 steps take
// one per step, the rolled steps and the wide stage offsets one per stage).
// Cody & Waite's reduction (Software Manual for the Elementary Functions,
// 1980): x = k pi/2 + r with k the integer nearest x 2/pi (added to and taken
// from 1.5 2^52, whose last bits then hold k) and r = (x - k P1) - k P2,
// pi/2 = P1 + P2 + O(1e-33), P1 the double nearest pi/2; |r| <= pi/4 up to
// the rounding of x 2/pi.  Then the Taylor series in z = r^2,
//   sin r = r - r^3/3! + ... + r^17/17!,  cos r = 1 - r^2/2! + ... + r^16/16!
// (first omitted terms below 1e-19 and 3e-18 for |r| <= pi/4), and the
// quadrant k mod 4 by swapping the two and flipping sign bits on the integer
// pipe.  Error: within one unit of 2^-52 absolute against a long-double
// reference over x in [-2, 4] and next to the multiples of pi/2 (2e7 draws);
// sin(-0) is +0.  |x| >= 2^10 (stage angles of a ray thrown through the
// polar axis, non-finite x) goes to CUDA's sincos, which reduces any
// argument exactly and so keeps such a ray's later arithmetic that of the
// library's sincos.  Coefficients in the full-rate operand form (vreg with a
// zero taken from x's bits and b.nz, formed next to each use).  FP32: sincosf.
template <typename T>
struct Trig;
template <>
struct Trig<double> {
  __device__ __forceinline__ static void sc(const BH<double>& b, double x, double* s, double* c) {
    if ((__double2hiint(x) & 0x7fffffff) >= 0x40900000) {  // |x| >= 2^10, inf, NaN
      sincos(x, s, c);
      return;
    }
    const unsigned long long vz =
        (unsigned long long)__double_as_longlong(x) & ((unsigned long long)__double_as_longlong(b.nz) & 0x7fffffffffffffffull);
    auto K = [&](double v) { return vreg(v, vz); };
    const double t = fma(x, K(0x1.45f306dc9c883p-1), K(0x1.8p52));
    const double kd = fma(t, b.one, K(-0x1.8p52));
    const unsigned q = (unsigned)__double2loint(t);
    double r = fma(-kd, K(0x1.921fb54442d18p+0), x);
    r = fma(-kd, K(0x1.1a62633145c07p-54), r);
    const double z = vmul(b, r, r);
    double p = fma(z, K(1.0 / 355687428096000.0), K(-1.0 / 1307674368000.0));
    p = fma(z, p, K(1.0 / 6227020800.0));
    p = fma(z, p, K(-1.0 / 39916800.0));
    p = fma(z, p, K(1.0 / 362880.0));
    p = fma(z, p, K(-1.0 / 5040.0));
    p = fma(z, p, K(1.0 / 120.0));
    p = fma(z, p, K(-1.0 / 6.0));
    const double sr = fma(vmul(b, r, z), p, r);
    double pc = fma(z, K(1.0 / 20922789888000.0), K(-1.0 / 87178291200.0));
    pc = fma(z, pc, K(1.0 / 479001600.0));
    pc = fma(z, pc, K(-1.0 / 3628800.0));
    pc = fma(z, pc, K(1.0 / 40320.0));
    pc = fma(z, pc, K(-1.0 / 720.0));
    pc = fma(z, pc, K(1.0 / 24.0));
    pc = fma(z, pc, -b.half);
    const double cr = fma(z, pc, b.one);
    const unsigned long long bs = (q & 1u) ? __double_as_longlong(cr) : __double_as_longlong(sr);
    const unsigned long long bc = (q & 1u) ? __double_as_longlong(sr) : __double_as_longlong(cr);
    *s = __longlong_as_double((long long)(bs ^ ((unsigned long long)(q & 2u) << 62)));
    *c = __longlong_as_double((long long)(bc ^ ((unsigned long long)((q + 1u) & 2u) << 62)));
  }
};
template <>
struct Trig<float> {
  __device__ __forceinline__ static void sc(const BH<float>&, float x, float* s, float* c) { sincosf(x, s, c); }
};

// sin and cos at a stage angle th = th0 + c x (c x = d, the stage's offset
// from the step's start angle th0), given s0 = sin th0 and c0 = cos th0.
// FP64 with |d| < 1/4: the angle-addition formulas with sin d and cos d - 1
// from their Taylor series,
//   sin d = d - d^3/3! + ... - d^11/11!,  cos d - 1 = -d^2/2! + ... + d^12/12!
// (the first omitted terms are below 1e-17 relative for |d| <= 1/4), and for
// |d| < 2^-5 the shorter
//   sin d = d - d^3/3! + d^5/5! - d^7/7!,  cos d - 1 = -d^2/2! + ... + d^8/8!
// (first omitted terms below 1e-19 absolute there), so one sincos serves the
// four stages of a step; th itself is formed only for the sincos taken when
// |d| >= 1/4.  Otherwise, and in FP32: sincos of th = fma(c, x, th0).  The
// tier is a per-lane choice on the bits of d, so a ray's result never depends
// on the other rays of its warp.
template <typename T>
__device__ __forceinline__ void stage_trig(const BH<T>& b, T s0, T c0, T c, T x, T th0, T* s, T* cs) {
  Trig<T>::sc(b, fma(c, x, th0), s, cs);
}
// The range tests read the exponent bits on the integer pipe (an FP64 compare
// would take an issue of the FP64 unit, which costs as much as an FMA there);
// sin th = s0 + c0 sin d + s0 (cos d - 1) and likewise cos th are two FMAs
// each.  Products and coefficients in the full-rate operand forms (vmul).
template <>
__device__ __forceinline__ void stage_trig<double>(const BH<double>& b, double s0, double c0, double c, double x,
                                                   double th0, double* s, double* cs) {
  const double* k = b.k;  // k[n - 3] = 1/n!
  const double d = vmul(b, c, x);
  const int ex = __double2hiint(d) & 0x7fffffff;
  double sd, cm1;
  if (ex < 0x3fa00000) {  // |d| < 2^-5
    const double z = vmul(b, d, d);
    double ps = fma(z, -k[4], k[2]);
    ps = fma(z, ps, -k[0]);
    sd = fma(vmul(b, d, z), ps, d);
    double pc = fma(z, k[5], -k[3]);
    pc = fma(z, pc, k[1]);
    pc = fma(z, pc, -b.half);
    cm1 = vmul(b, z, pc);
  } else if (ex < 0x3fd00000) {  // |d| < 1/4 (NaN: no)
    const double z = vmul(b, d, d);
    double ps = fma(z, -k[8], k[6]);
    ps = fma(z, ps, -k[4]);
    ps = fma(z, ps, k[2]);
    ps = fma(z, ps, -k[0]);
    sd = fma(vmul(b, d, z), ps, d);
    double pc = fma(z, k[9], -k[7]);
    pc = fma(z, pc, k[5]);
    pc = fma(z, pc, -k[3]);
    pc = fma(z, pc, k[1]);
    pc = fma(z, pc, -b.half);
    cm1 = vmul(b, z, pc);
  } else {
    Trig<double>::sc(b, fma(c, x, th0), s, cs);
    return;
  }
  *s = fma(s0, cm1, fma(c0, sd, s0));
  *cs = fma(c0, cm1, fma(-s0, sd, c0));
}

// 2x for a finite, normal x: the exponent field raised by one, on the integer
// pipe (exact; an FP64 add or multiply would take an issue of the FP64 unit).
// Used for 2r and 4r of stage radii, which are finite and normal on every ray
// still traced: r = 0 (which this maps to the smallest normal number) lies
// inside the capture radius, and a non-finite r makes the whole state
// non-finite, so either ray ends at this step.  FP32: x + x.
__device__ __forceinline__ double twice(double x) {
  return __hiloint2double(__double2hiint(x) + 0x00100000, __double2loint(x));
}
__device__ __forceinline__ float twice(float x) { return x + x; }

// Ordering key of a radius for the termination tests, on the integer pipe:
// the signed 64-bit view of its bits, with every NaN mapped above all
// numbers.  For r_ref > 0 finite and any r: key(r) <= bits(r_ref) exactly
// when r <= r_ref holds in IEEE arithmetic, and key(r) >= bits(r_ref)
// exactly when r >= r_ref or r is NaN (termination tests non-finite states
// before escape, so the NaN case never decides an escape).  The minimum of
// several keys is <= bits(r_ref) exactly when one of the radii is <= r_ref.
__device__ __forceinline__ long long radius_key(double r) {
  const long long b = __double_as_longlong(r);
  return (b & 0x7fffffffffffffffll) > 0x7ff0000000000000ll ? 0x7ff8000000000000ll : b;
}
__device__ __forceinline__ bool key_le(long long k, double ref) { return k <= __double_as_longlong(ref); }
__device__ __forceinline__ bool key_ge(long long k, double ref) { return k >= __double_as_longlong(ref); }

// ---------------------------------------------------------------------------
// Schwarzschild: Gamma^t_tr = M/(r f), Gamma^r_tt = M f / r^3,
// Gamma^r_rr = -M/(r f), Gamma^r_thth = -f, Gamma^r_phph = -f sin^2,
// Gamma^th_rth = Gamma^ph_rph = 1/r, Gamma^th_phph = -sin cos,
// Gamma^ph_thph = cot, with f = r - 2M.
template <typename T, bool kFastRcp = true>
__device__ __forceinline__ void accel_schw(const BH<T>& bh, T r, T s, T c, T ut, T ur, T uth, T uph,
                                           T acc[4]) {
  auto mul = [&](T x, T y) { return vmul<T>(bh, x, y); };
  const T f = vsub<T>(bh, r, bh.twoM);
  const T rf = mul(r, f);
  const T den = mul(rf, s);
  const T inv = kFastRcp ? recip<T>(den, bh.one) : T(1) / den;  // 1 / (r f sin)
  const T ir = mul(mul(f, s), inv);       // 1/r
  const T i_f = mul(mul(r, s), inv);      // 1/f
  const T cot = mul(mul(c, rf), inv);     // cos/sin
  const T Mirf = mul(mul(bh.M, ir), i_f); // M/(r f)
  const T ang = fma(mul(mul(s, s), uph), uph, mul(uth, uth));
  acc[0] = mul(mul(mul(-bh.two, Mirf), ut), ur);
  acc[1] = fma(f, ang, fma(mul(Mirf, ur), ur, mul(mul(-mul(mul(mul(mul(bh.M, f), ir), ir), ir), ut), ut)));
  acc[2] = fma(mul(mul(s, c), uph), uph, mul(mul(mul(-bh.two, ir), ur), uth));
  acc[3] = mul(mul(-bh.two, uph), fma(ir, ur, mul(cot, uth)));
}

// ---------------------------------------------------------------------------
// Kerr (see the file header).  With q = 2Mr/rho^2 the metric is
//   g_tt = q - 1, g_tph = -a s^2 q, g_phph = s^2 (r^2 + a^2) + a^2 s^4 q,
//   g_rr = rho^2/Delta, g_thth = rho^2,
//   d_r q = (2M - 2 r q)/rho^2, d_th q = 2 a^2 s c q / rho^2,
// and q enters the (t, phi) block only through g_tt u^t u^t + 2 g_tph u^t u^ph
// + g_phph u^ph u^ph = (q - 1)(u^t)^2 + ... whose q-part is q v^2 with
// v = u^t - a s^2 u^ph.  Collecting terms of the first-kind contraction
// W_nu = (d_a g_{nu b}) u^a u^b - 1/2 (d_nu g_ab) u^a u^b, D = u^r d_r + u^th d_th:
//   W_t = (D q) v - 2 a q s c u^th u^ph,
//   X = a s^2 W_t + W_ph = 2 s c u^th B + 2 r s^2 u^r u^ph,  B = (r^2 + a^2) u^ph - a q v
//   (the D q terms cancel in X),
//   2 W_r = (u^r)^2 d_r g_rr + 2 u^r u^th d_th g_rr - K_r,
//   K_r = (d_r q) v^2 + 2 r (s^2 (u^ph)^2 + (u^th)^2),
//   2 W_th = 4 r u^r u^th - 2 a^2 s c (u^th)^2 - K_th,
//   K_th = (d_th q) v^2 + 2 s c u^ph (B - a q v) + (d_th g_rr) (u^r)^2,
// and acc^mu = -g^{mu nu} W_nu with g^tt = -(r^2 + a^2 + a^2 s^2 q)/Delta,
// g^tph = -a q/Delta, g^phph = (1 - q)/(Delta s^2), g^rr = Delta/rho^2,
// g^thth = 1/rho^2:
//   acc^t = ((r^2 + a^2) W_t + a q X) / Delta,  acc^ph = ((q - 1) X + a s^2 W_t) / (Delta s^2),
//   acc^r = -Delta W_r / rho^2,                  acc^th = -W_th / rho^2.
// The same bilinear form as the twenty second-kind symbols of BL Kerr, in 71
// FP64 operations plus one reciprocal.
// Products and sums in the full-rate FP64 operand forms (vmul, vadd, vsub:
// the same IEEE results).
template <typename T, bool kFastRcp = true>
__device__ __forceinline__ void accel_kerr(const BH<T>& bh, T r, T s, T c, T ut, T ur, T uth, T uph,
                                           T acc[4]) {
  auto mul = [&](T x, T y) { return vmul<T>(bh, x, y); };
  auto add = [&](T x, T y) { return vadd<T>(bh, x, y); };
  auto sub = [&](T x, T y) { return vsub<T>(bh, x, y); };
  const T a = bh.a, a2 = bh.a2;
  const T s2 = mul(s, s), sc = mul(s, c);
  const T r2a2 = fma(r, r, a2);
  const T rho2 = fma(-a2, s2, r2a2);
  const T tMr = mul(bh.twoM, r);
  const T Delta = sub(r2a2, tMr);
  const T Ds2 = mul(Delta, s2);
  const T den = mul(rho2, Ds2);
  const T inv = kFastRcp ? recip<T>(den, bh.one) : T(1) / den;
  const T irho2 = mul(Ds2, inv);
  const T iDs2 = mul(rho2, inv);  // 1 / (Delta sin^2)
  const T iDelta = mul(iDs2, s2);
  const T q = mul(tMr, irho2);
  const T r_2 = twice(r);
  const T dq_r = mul(fma(-r_2, q, bh.twoM), irho2);
  const T a2sc2 = mul(bh.two_a2, sc);  // 2 a^2 sin cos
  const T dq_th = mul(a2sc2, mul(q, irho2));
  const T Dq = fma(ur, dq_r, mul(uth, dq_th));
  const T as2 = mul(a, s2);
  const T v = fma(-as2, uph, ut);
  const T aq = mul(a, q);
  const T aqv = mul(aq, v);
  const T B = fma(r2a2, uph, -aqv);
  const T sc2 = add(sc, sc);
  const T sc2uth = mul(sc2, uth);
  const T X = fma(sc2uth, B, mul(mul(r_2, s2), mul(ur, uph)));
  const T Wt = fma(Dq, v, mul(-mul(aq, sc2uth), uph));
  acc[0] = mul(fma(r2a2, Wt, mul(aq, X)), iDelta);
  acc[3] = mul(fma(q, X, fma(as2, Wt, -X)), iDs2);
  const T v2 = mul(v, v);
  const T Kr = fma(dq_r, v2, mul(r_2, fma(mul(s2, uph), uph, mul(uth, uth))));
  const T drr_r = mul(fma(mul(-sub(r_2, bh.twoM), rho2), iDelta, r_2), iDelta);  // d_r g_rr
  const T drr_th = mul(-a2sc2, iDelta);                                             // d_th g_rr
  const T Wr2 = fma(ur, fma(ur, drr_r, mul(add(uth, uth), drr_th)), -Kr);           // 2 W_r
  const T Kth = fma(dq_th, v2, fma(mul(sc2, uph), sub(B, aqv), mul(drr_th, mul(ur, ur))));
  const T Wth2 = fma(uth, fma(-a2sc2, uth, mul(twice(r_2), ur)), -Kth);            // 2 W_th
  const T hirho2 = mul(bh.half, irho2);
  acc[1] = mul(-Wr2, mul(Delta, hirho2));
  acc[2] = mul(-Wth2, hirho2);
}

// The acceleration at (r, theta) given s = sin theta, c = cos theta
// (kFastRcp: the refined hardware reciprocal in FP64, else the division).
template <bool kKerr, typename T, bool kFastRcp = true>
__device__ __forceinline__ void accel_sc(const BH<T>& bh, T r, T s, T c, T ut, T ur, T uth, T uph, T acc[4]) {
  if (kKerr)
    accel_kerr<T, kFastRcp>(bh, r, s, c, ut, ur, uth, uph, acc);
  else
    accel_schw<T, kFastRcp>(bh, r, s, c, ut, ur, uth, uph, acc);
}

template <bool kKerr, typename T>
__device__ __forceinline__ void accel(const BH<T>& bh, T r, T th, T ut, T ur, T uth, T uph, T acc[4]) {
  T s, c;
  Trig<T>::sc(bh, th, &s, &c);
  accel_sc<kKerr, T>(bh, r, s, c, ut, ur, uth, uph, acc);
}

// ---------------------------------------------------------------------------
// One classical RK4 step (tableau c = (0, 1/2, 1/2, 1), b = (1, 2, 2, 1)/6)
// of y = (x, u).  t and phi never enter the right-hand side, so their stage
// values are not formed.  The weighted sums k1 + 2 k2 + 2 k3 + k4 of the
// stage velocities and accelerations are accumulated stage by stage (the same
// operations in the same order whether the stage loop is unrolled or not, so
// both forms give the same bits).  kRolled keeps one copy of the right-hand
// side in the code (the FP32_MIXED kernels, whose size otherwise costs
// instruction-cache misses; there each stage takes its own sincos and the
// division, which keeps those kernels' register count down: their FP64 steps
// are rare and their occupancy matters more).  Returns the smallest radius
// among the three intermediate stage points (used by the capture test; NaN
// radii are passed over).  FP64 unrolled: the minimum is taken over
// radius_key on the integer pipe and the radius returned is the one whose
// key is smallest, which decides "some stage radius <= r_cap" identically.
template <bool kKerr, typename T, bool kRolled = false>
__device__ __forceinline__ T rk4_step(const BH<T>& bh, T h, T y[8]) {
  constexpr bool kKeys = sizeof(T) == 8 && !kRolled;
  const T hh = vmul<T>(bh, bh.half, h);
  T r = y[1], th = y[2];
  T u[4] = {y[4], y[5], y[6], y[7]};
  T sx[4], su[4];
  T rmin = T(0);
  long long kmin = 0;
  T s0 = T(0), c0 = T(1);
  if constexpr (!kRolled) Trig<T>::sc(bh, y[2], &s0, &c0);
  T sn = s0, cs = c0;
  auto stage = [&](int s) {
    T acc[4];
    if constexpr (kRolled) {
      T sr, cr;
      Trig<T>::sc(bh, th, &sr, &cr);
      accel_sc<kKerr, T, false>(bh, r, sr, cr, u[0], u[1], u[2], u[3], acc);
    } else {
      accel_sc<kKerr, T>(bh, r, sn, cs, u[0], u[1], u[2], u[3], acc);
    }
    if (s == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        sx[j] = u[j];
        su[j] = acc[j];
      }
    } else {
      const T w = s == 3 ? bh.one : bh.two;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        sx[j] = fma(w, u[j], sx[j]);
        su[j] = fma(w, acc[j], su[j]);
      }
    }
    if (s < 3) {
      const T c = s < 2 ? hh : h;
      r = fma(c, u[1], y[1]);
      if constexpr (kRolled)
        th = fma(c, u[2], y[2]);
      else
        stage_trig<T>(bh, s0, c0, c, u[2], y[2], &sn, &cs);
#pragma unroll
      for (int j = 0; j < 4; ++j) u[j] = fma(c, acc[j], y[4 + j]);
      if constexpr (kKeys) {
        const long long k = radius_key(r);
        kmin = s == 0 ? k : min(kmin, k);
      } else {
        rmin = s == 0 ? r : fmin(rmin, r);
      }
    }
  };
  if constexpr (kRolled) {
#pragma unroll 1
    for (int s = 0; s < 4; ++s) stage(s);
  } else {
#pragma unroll
    for (int s = 0; s < 4; ++s) stage(s);
  }
  const T h6 = vmul<T>(bh, h, bh.k[0]);  // h/6
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    y[j] = fma(h6, sx[j], y[j]);
    y[4 + j] = fma(h6, su[j], y[4 + j]);
  }
  if constexpr (kKeys) rmin = __longlong_as_double(kmin);
  return rmin;
}

// ---------------------------------------------------------------------------
// Canonical form (Sec. 2, eq. Ham): state z = (x^mu, p_mu), dx^mu/dl =
// dH/dp_mu, dp_mu/dl = -dH/dx^mu with H = g^{ab} p_a p_b / 2.  For Kerr in BL
// coordinates, with P = (r^2 + a^2) p_t + a p_ph and T = p_ph + a s^2 p_t,
//   2 rho^2 H = F = Delta p_r^2 + p_th^2 - P^2 / Delta + T^2 / s^2,
// so dx/dl follows from dF/dp and dp_r/dl = -(dF/dr - F d(rho^2)/dr / rho^2)
// / (2 rho^2), dp_th/dl likewise; p_t and p_ph are constant (H does not
// depend on t, ph) and are not integrated.  f = (dt, dr, dth, dph, dp_r,
// dp_th)/dl.  One reciprocal, as in the geodesic form.
// Products and sums in the full-rate FP64 operand forms (vmul, vadd, vsub).
template <typename T, bool kFastRcp = true>
__device__ __forceinline__ void ham_kerr(const BH<T>& bh, T r, T s, T c, T pt, T pr, T pth, T pph, T f[6]) {
  auto mul = [&](T x, T y) { return vmul<T>(bh, x, y); };
  auto sub = [&](T x, T y) { return vsub<T>(bh, x, y); };
  const T a = bh.a, a2 = bh.a2;
  const T s2 = mul(s, s), sc = mul(s, c);
  const T rho2 = fma(a2, mul(c, c), mul(r, r));
  const T Delta = fma(r, sub(r, bh.twoM), a2);
  const T rD = mul(rho2, Delta);
  const T den = mul(rD, s2);
  const T inv = kFastRcp ? recip<T>(den, bh.one) : T(1) / den;
  const T irho2 = mul(mul(Delta, s2), inv);
  const T iDelta = mul(mul(rho2, s2), inv);
  const T is2 = mul(rD, inv);
  const T r2a2 = fma(r, r, a2);
  const T P = fma(r2a2, pt, mul(a, pph));
  const T Tq = fma(mul(a, s2), pt, pph);
  const T PiD = mul(P, iDelta);
  const T TiS = mul(Tq, is2);
  f[0] = mul(fma(-r2a2, PiD, mul(a, Tq)), irho2);
  f[1] = mul(mul(Delta, pr), irho2);
  f[2] = mul(pth, irho2);
  f[3] = mul(fma(-a, PiD, TiS), irho2);
  const T pr2 = mul(pr, pr);
  const T F = fma(Tq, TiS, fma(-P, PiD, fma(pth, pth, mul(Delta, pr2))));
  const T m4r = -twice(twice(r));  // -4 r
  const T dFr = fma(mul(bh.two, sub(r, bh.M)), fma(PiD, PiD, pr2), mul(mul(m4r, pt), PiD));
  const T dFth = mul(mul(mul(bh.two, mul(sc, is2)), Tq), fma(mul(bh.two, a), pt, -TiS));
  const T mh = mul(-bh.half, irho2);
  f[4] = mul(mh, fma(mul(mul(-bh.two, r), F), irho2, dFr));
  f[5] = mul(mh, fma(mul(mul(bh.two_a2, sc), F), irho2, dFth));
}

// ---------------------------------------------------------------------------
// 3+1 form (Sec. 2, eq. ADM and the free-particle Lagrangian, then eq. Ham):
// the same canonical state z = (x^mu, p_mu), with H written through the lapse
// alpha, the shift beta^i and the spatial metric gamma_ij instead of
// g^{mu nu} of eq. kerr.  The right-hand side below holds for any
// stationary, axisymmetric, circular spacetime: every function depends on r
// and theta only, beta^i = (0, 0, beta^ph) and gamma_ij is diagonal.  Kerr in
// BL coordinates (Sec. 2, the comparison of eq. ADM with eq. kerr) is one
// such metric; numerically computed metrics of rotating compact objects are
// others.  A metric enters only through an Adm<T> point filled by a provider
// function of (r, theta).  With A = p_t - beta^ph p_ph,
//   H = -A^2 / (2 alpha^2) + (p_r^2/g_rr + p_th^2/g_thth + p_ph^2/g_phph) / 2
// (g_ii standing for gamma_ii), so
//   dt/dl = -A/alpha^2,  dr/dl = p_r/g_rr,  dth/dl = p_th/g_thth,
//   dph/dl = p_ph/g_phph + beta^ph A/alpha^2,
//   dp_k/dl = -(A/alpha^2) (p_ph d_k beta^ph + A d_k ln alpha)
//             + 1/2 sum_i (p_i^2/g_ii) d_k ln g_ii        (k = r, theta),
// and p_t, p_ph are constant.
enum HamForm { kHamKerrBL = 1, kHamAdm = 2 };

template <typename T>
struct Adm {
  T alpha2, beta, gam[3];  // alpha^2, beta^ph, gamma_rr, gamma_thth, gamma_phph
  T ialpha2, igam[3];      // 1/alpha^2, 1/gamma_ii
  T dlna[2];               // d_r ln alpha, d_th ln alpha
  T dbeta[2];              // d_r beta^ph, d_th beta^ph
  T dlng[3][2];            // d_k ln gamma_ii
};

// Provider: Kerr's lapse, shift and 3-metric in BL coordinates,
//   alpha^2 = rho^2 Delta / Sigma, beta^ph = -2 M a r / Sigma,
//   gamma = diag(rho^2/Delta, rho^2, Sigma sin^2 / rho^2),
// with the logarithmic derivatives of rho^2, Delta, Sigma (d_r rho^2 = 2r,
// d_th rho^2 = -2 a^2 s c, d_r Delta = 2(r - M), d_r Sigma = 4 r (r^2 + a^2)
// - a^2 s^2 d_r Delta, d_th Sigma = -2 a^2 Delta s c).  FP64 shares one
// division among 1/rho^2, 1/Delta, 1/Sigma and 1/sin^2; FP32 takes 1/Sigma
// apart (the product of all four would overflow near r = 10^4).
template <typename T, bool kFastRcp = true>
__device__ __forceinline__ void adm_kerr_sc(const BH<T>& bh, T r, T s, T c, Adm<T>& m) {
  auto mul = [&](T x, T y) { return vmul<T>(bh, x, y); };
  auto add = [&](T x, T y) { return vadd<T>(bh, x, y); };
  auto sub = [&](T x, T y) { return vsub<T>(bh, x, y); };
  const T a2 = bh.a2;
  const T s2 = mul(s, s), sc = mul(s, c);
  const T rho2 = fma(a2, mul(c, c), mul(r, r));
  const T Delta = fma(r, sub(r, bh.twoM), a2);
  const T r2a2 = fma(r, r, a2);
  const T Sigma = fma(r2a2, r2a2, mul(-mul(a2, Delta), s2));
  const T rD = mul(rho2, Delta);
  T irho2, iDelta, iSigma, is2;
  if constexpr (sizeof(T) == 8) {
    const T SS = mul(Sigma, s2);
    const T den = mul(rD, SS);
    const T inv = kFastRcp ? recip<T>(den, bh.one) : T(1) / den;
    irho2 = mul(mul(Delta, SS), inv);
    iDelta = mul(mul(rho2, SS), inv);
    iSigma = mul(mul(rD, s2), inv);
    is2 = mul(mul(rD, Sigma), inv);
  } else {
    const T inv = T(1) / (rD * s2);
    irho2 = Delta * s2 * inv;
    iDelta = rho2 * s2 * inv;
    is2 = rD * inv;
    iSigma = T(1) / Sigma;
  }
  m.alpha2 = mul(rD, iSigma);
  m.ialpha2 = mul(mul(Sigma, irho2), iDelta);
  const T m2Ma = mul(-bh.twoM, bh.a);  // -2 M a
  m.beta = mul(mul(m2Ma, r), iSigma);
  m.gam[0] = mul(rho2, iDelta);
  m.gam[1] = rho2;
  m.gam[2] = mul(mul(Sigma, s2), irho2);
  m.igam[0] = mul(Delta, irho2);
  m.igam[1] = irho2;
  m.igam[2] = mul(mul(rho2, iSigma), is2);
  const T a2sc2 = mul(bh.two_a2, sc);
  const T lrho_r = mul(twice(r), irho2), lrho_t = mul(-a2sc2, irho2);
  const T dDr = mul(bh.two, sub(r, bh.M));
  const T lD_r = mul(dDr, iDelta);
  const T lS_r = mul(fma(twice(twice(r)), r2a2, mul(-mul(a2, s2), dDr)), iSigma);
  const T lS_t = mul(mul(-a2sc2, Delta), iSigma);
  m.dlna[0] = mul(bh.half, sub(add(lrho_r, lD_r), lS_r));
  m.dlna[1] = mul(bh.half, sub(lrho_t, lS_t));
  m.dbeta[0] = fma(-m.beta, lS_r, mul(m2Ma, iSigma));
  m.dbeta[1] = mul(-m.beta, lS_t);
  m.dlng[0][0] = sub(lrho_r, lD_r);
  m.dlng[0][1] = lrho_t;
  m.dlng[1][0] = lrho_r;
  m.dlng[1][1] = lrho_t;
  m.dlng[2][0] = sub(lS_r, lrho_r);
  m.dlng[2][1] = fma(mul(bh.two, sc), is2, sub(lS_t, lrho_t));
}

template <typename T>
__device__ __forceinline__ void adm_kerr(const BH<T>& bh, T r, T th, Adm<T>& m) {
  T s, c;
  Trig<T>::sc(bh, th, &s, &c);
  adm_kerr_sc<T>(bh, r, s, c, m);
}

// The 3+1 right-hand side f = (dt, dr, dth, dph, dp_r, dp_th)/dl at one
// point of any provider (formulas above).
template <typename T>
__device__ __forceinline__ void adm_rhs(const BH<T>& bh, const Adm<T>& m, T pt, T pr, T pth, T pph, T f[6]) {
  auto mul = [&](T x, T y) { return vmul<T>(bh, x, y); };
  const T A = fma(-m.beta, pph, pt);
  const T u = mul(A, m.ialpha2);
  const T vr = mul(pr, m.igam[0]), vth = mul(pth, m.igam[1]), vph = mul(pph, m.igam[2]);
  f[0] = -u;
  f[1] = vr;
  f[2] = vth;
  f[3] = fma(m.beta, u, vph);
  const T qr = mul(mul(bh.half, pr), vr), qth = mul(mul(bh.half, pth), vth), qph = mul(mul(bh.half, pph), vph);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const T kin = fma(qph, m.dlng[2][k], fma(qth, m.dlng[1][k], mul(qr, m.dlng[0][k])));
    f[4 + k] = fma(-u, fma(pph, m.dbeta[k], mul(A, m.dlna[k])), kin);
  }
}

// The canonical right-hand side of one form: eq. Ham through g^{mu nu} of
// eq. kerr (kHamKerrBL) or through the 3+1 quantities of Kerr (kHamAdm).
template <int kForm, typename T, bool kFastRcp = true>
__device__ __forceinline__ void ham_rhs_sc(const BH<T>& bh, T r, T s, T c, T pt, T pr, T pth, T pph, T f[6]) {
  if constexpr (kForm == kHamAdm) {
    Adm<T> m;
    adm_kerr_sc<T, kFastRcp>(bh, r, s, c, m);
    adm_rhs<T>(bh, m, pt, pr, pth, pph, f);
  } else {
    ham_kerr<T, kFastRcp>(bh, r, s, c, pt, pr, pth, pph, f);
  }
}

template <int kForm, typename T>
__device__ __forceinline__ void ham_rhs(const BH<T>& bh, T r, T th, T pt, T pr, T pth, T pph, T f[6]) {
  T s, c;
  Trig<T>::sc(bh, th, &s, &c);
  ham_rhs_sc<kForm, T>(bh, r, s, c, pt, pr, pth, pph, f);
}

// p_mu = g_{mu nu} u^nu from the 3+1 quantities: g_tt = -alpha^2 +
// gamma_phph beta^2, g_tph = gamma_phph beta, g_ii = gamma_ii.
__device__ __forceinline__ void adm_lower(const Adm<double>& m, const double u[4], double p[4]) {
  const double w = m.gam[2] * fma(m.beta, u[0], u[3]);  // gamma_phph (beta u^t + u^ph)
  p[0] = fma(-m.alpha2, u[0], m.beta * w);
  p[1] = m.gam[0] * u[1];
  p[2] = m.gam[1] * u[2];
  p[3] = w;
}

// u^mu = g^{mu nu} p_nu from the 3+1 quantities (the first half of adm_rhs).
__device__ __forceinline__ void adm_raise(const Adm<double>& m, const double p[4], double u[4]) {
  double f[6];
  adm_rhs<double>(make_bh<double>(1.0, 0.0), m, p[0], p[1], p[2], p[3], f);
#pragma unroll
  for (int j = 0; j < 4; ++j) u[j] = f[j];
}

// One classical RK4 step of the canonical state z (same tableau and the same
// stage-by-stage sums as rk4_step); p_t = z[4] and p_ph = z[7] stay fixed.
// Returns the smallest radius among the three intermediate stage points (as
// rk4_step, by radius_key in the FP64 unrolled case).
template <typename T, bool kRolled = false, int kForm = kHamKerrBL>
__device__ __forceinline__ T rk4_step_ham(const BH<T>& bh, T h, T z[8]) {
  constexpr bool kKeys = sizeof(T) == 8 && !kRolled;
  const T hh = vmul<T>(bh, bh.half, h);
  T r = z[1], th = z[2], pr = z[5], pth = z[6];
  T sx[6];
  T rmin = T(0);
  long long kmin = 0;
  T s0 = T(0), c0 = T(1);
  if constexpr (!kRolled) Trig<T>::sc(bh, z[2], &s0, &c0);
  T sn = s0, cs = c0;
  auto stage = [&](int s) {
    T f[6];
    if constexpr (kRolled) {
      T sr, cr;
      Trig<T>::sc(bh, th, &sr, &cr);
      ham_rhs_sc<kForm, T, false>(bh, r, sr, cr, z[4], pr, pth, z[7], f);
    } else {
      ham_rhs_sc<kForm, T>(bh, r, sn, cs, z[4], pr, pth, z[7], f);
    }
    if (s == 0) {
#pragma unroll
      for (int j = 0; j < 6; ++j) sx[j] = f[j];
    } else {
      const T w = s == 3 ? bh.one : bh.two;
#pragma unroll
      for (int j = 0; j < 6; ++j) sx[j] = fma(w, f[j], sx[j]);
    }
    if (s < 3) {
      const T c = s < 2 ? hh : h;
      r = fma(c, f[1], z[1]);
      if constexpr (kRolled)
        th = fma(c, f[2], z[2]);
      else
        stage_trig<T>(bh, s0, c0, c, f[2], z[2], &sn, &cs);
      pr = fma(c, f[4], z[5]);
      pth = fma(c, f[5], z[6]);
      if constexpr (kKeys) {
        const long long k = radius_key(r);
        kmin = s == 0 ? k : min(kmin, k);
      } else {
        rmin = s == 0 ? r : fmin(rmin, r);
      }
    }
  };
  if constexpr (kRolled) {
#pragma unroll 1
    for (int s = 0; s < 4; ++s) stage(s);
  } else {
#pragma unroll
    for (int s = 0; s < 4; ++s) stage(s);
  }
  const T h6 = vmul<T>(bh, h, bh.k[0]);  // h/6
#pragma unroll
  for (int j = 0; j < 4; ++j) z[j] = fma(h6, sx[j], z[j]);
  z[5] = fma(h6, sx[4], z[5]);
  z[6] = fma(h6, sx[5], z[6]);
  if constexpr (kKeys) rmin = __longlong_as_double(kmin);
  return rmin;
}

// p_mu = g_{mu nu} u^nu (Kerr, BL): the canonical momenta of a state.
__device__ __forceinline__ void lower_velocity(double M, double a, const double y[8], double p[4]) {
  double s, c;
  sincos(y[2], &s, &c);
  const double r = y[1], a2 = a * a, s2 = s * s;
  const double rho2 = fma(a2, c * c, r * r);
  const double Delta = fma(r, r - 2.0 * M, a2);
  const double q = 2.0 * M * r / rho2;
  const double gtp = -a * s2 * q;
  const double gpp = s2 * fma(a2 * s2, q, fma(r, r, a2));
  p[0] = fma(q - 1.0, y[4], gtp * y[7]);
  p[1] = rho2 / Delta * y[5];
  p[2] = rho2 * y[6];
  p[3] = fma(gtp, y[4], gpp * y[7]);
}

// u^mu = g^{mu nu} p_nu (Kerr, BL); the (t, ph) block inverse has
// determinant -Delta sin^2.
__device__ __forceinline__ void raise_momentum(double M, double a, const double z[8], double u[4]) {
  double s, c;
  sincos(z[2], &s, &c);
  const double r = z[1], a2 = a * a, s2 = s * s;
  const double rho2 = fma(a2, c * c, r * r);
  const double Delta = fma(r, r - 2.0 * M, a2);
  const double q = 2.0 * M * r / rho2;
  const double gtt = q - 1.0;
  const double gtp = -a * s2 * q;
  const double gpp = s2 * fma(a2 * s2, q, fma(r, r, a2));
  const double det = -Delta * s2;
  u[0] = fma(gpp, z[4], -gtp * z[7]) / det;
  u[1] = Delta / rho2 * z[5];
  u[2] = z[6] / rho2;
  u[3] = fma(gtt, z[7], -gtp * z[4]) / det;
}

// ---------------------------------------------------------------------------
// Conserved quantities in FP64: p = g u; E = -p_t, L_z = p_ph,
// Q = p_th^2 + cos^2 (a^2 (mu^2 - E^2) + L_z^2 / sin^2) with mu^2 = -g(u,u),
// norm = g(u,u).
__device__ __forceinline__ void invariants64(double M, double a, const double y[8], double inv[4]) {
  double s, c;
  sincos(y[2], &s, &c);
  const double r = y[1], a2 = a * a, s2 = s * s;
  const double rho2 = fma(a2, c * c, r * r);
  const double Delta = fma(r, r - 2.0 * M, a2);
  const double q = 2.0 * M * r / rho2;
  const double gtt = q - 1.0;
  const double gtp = -a * s2 * q;
  const double gpp = s2 * fma(a2 * s2, q, fma(r, r, a2));
  const double pt = fma(gtt, y[4], gtp * y[7]);
  const double pp = fma(gtp, y[4], gpp * y[7]);
  const double pr = rho2 / Delta * y[5];
  const double pth = rho2 * y[6];
  const double norm = fma(pt, y[4], fma(pr, y[5], fma(pth, y[6], pp * y[7])));
  const double E = -pt;
  inv[0] = E;
  inv[1] = pp;
  inv[2] = fma(pth, pth, c * c * fma(a2, fma(-E, E, -norm), pp * pp / s2));
  inv[3] = norm;
}

}  // namespace malbec

namespace malbec {

// ---------------------------------------------------------------------------
// Dormand-Prince 5(4) (Dormand & Prince, J. Comput. Appl. Math. 6 (1980)
// 19-26), one of the further Runge-Kutta methods the paper's conclusions
// name: seven stages, the seventh taken at the fifth-order result, so that
// it is the first stage of the next step (k1 = k7 of the last accepted
// attempt).  One attempt of size h from y with k1 = f(y): y5 (fifth order),
// e = y5 - y4 (the embedded fourth-order result), k7 = f(y5); returns the
// smallest radius among the stage points 2..7.  One sincos per attempt: the
// stage angles are reached by stage_trig.  kForm: the geodesic form on
// y = (x, u), or a canonical form on z = (x, p), whose p_t and p_ph have zero
// derivative (their k components are 0, so they never change).
template <bool kKerr, int kForm = 0>
__device__ __forceinline__ double dopri5_attempt(const BH<double>& bh, double h, const double y[8],
                                                 const double k1[8], double y5[8], double e[8], double k7[8]) {
  double s0, c0;
  Trig<double>::sc(bh, y[2], &s0, &c0);
  // the tableau's coefficients as per-thread registers (full-rate DFMAs):
  // vreg with a zero that depends on this attempt's h, so that each is formed
  // next to its use instead of all 35 being held through the attempt
  const unsigned long long vzh =
      (unsigned long long)__double_as_longlong(h) & ((unsigned long long)__double_as_longlong(bh.nz) & 0x7fffffffffffffffull);
  auto K = [&](double c) { return vreg(c, vzh); };
  double k2[8], k3[8], k4[8], k5[8], k6[8];
  double d[8];
  double rmin = 0.0;
  // k = f(y + h d): stage velocity (the first half of k) and acceleration
  auto stage = [&](double k[8], bool first) {
    const double r = fma(h, d[1], y[1]);
    double sn, cs;
    stage_trig<double>(bh, s0, c0, h, d[2], y[2], &sn, &cs);
    if constexpr (kForm == 0) {
      // k = (u, -Gamma u u) at the stage point
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = fma(h, d[4 + j], y[4 + j]);
      accel_sc<kKerr, double>(bh, r, sn, cs, k[0], k[1], k[2], k[3], k + 4);
    } else {
      // k = (dH/dp, -dH/dx) at the stage point; p_t, p_ph stay y[4], y[7]
      double f[6];
      ham_rhs_sc<kForm, double>(bh, r, sn, cs, y[4], fma(h, d[5], y[5]), fma(h, d[6], y[6]), y[7], f);
#pragma unroll
      for (int j = 0; j < 4; ++j) k[j] = f[j];
      k[4] = 0.0;
      k[5] = f[4];
      k[6] = f[5];
      k[7] = 0.0;
    }
    rmin = first ? r : fmin(rmin, r);
  };
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = vmul(bh, K(1.0 / 5.0), k1[q]);
  stage(k2, true);
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = fma(K(3.0 / 40.0), k1[q], vmul(bh, K(9.0 / 40.0), k2[q]));
  stage(k3, false);
#pragma unroll
  for (int q = 0; q < 8; ++q) d[q] = fma(K(44.0 / 45.0), k1[q], fma(K(-56.0 / 15.0), k2[q], vmul(bh, K(32.0 / 9.0), k3[q])));
  stage(k4, false);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    d[q] = fma(K(19372.0 / 6561.0), k1[q],
               fma(K(-25360.0 / 2187.0), k2[q], fma(K(64448.0 / 6561.0), k3[q], vmul(bh, K(-212.0 / 729.0), k4[q]))));
  stage(k5, false);
#pragma unroll
  for (int q = 0; q < 8; ++q)
    d[q] = fma(K(9017.0 / 3168.0), k1[q],
               fma(K(-355.0 / 33.0), k2[q],
                   fma(K(46732.0 / 5247.0), k3[q], fma(K(49.0 / 176.0), k4[q], vmul(bh, K(-5103.0 / 18656.0), k5[q])))));
  stage(k6, false);
  // the fifth-order weights (a_2 = 0)
#pragma unroll
  for (int q = 0; q < 8; ++q)
    d[q] = fma(K(35.0 / 384.0), k1[q],
               fma(K(500.0 / 1113.0), k3[q],
                   fma(K(125.0 / 192.0), k4[q], fma(K(-2187.0 / 6784.0), k5[q], vmul(bh, K(11.0 / 84.0), k6[q])))));
#pragma unroll
  for (int q = 0; q < 8; ++q) y5[q] = fma(h, d[q], y[q]);
  stage(k7, false);
  // e = h sum_j (b_j - bhat_j) k_j
#pragma unroll
  for (int q = 0; q < 8; ++q)
    e[q] = vmul(bh, h, fma(K(71.0 / 57600.0), k1[q],
                   fma(K(-71.0 / 16695.0), k3[q],
                       fma(K(71.0 / 1920.0), k4[q],
                           fma(K(-17253.0 / 339200.0), k5[q],
                               fma(K(22.0 / 525.0), k6[q], vmul(bh, K(-1.0 / 40.0), k7[q])))))));
  return rmin;
}

// RMS error norm of an attempt with the scale atol + rtol max(|y|, |y5|)
// (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4), and the step-size
// factor that follows it: 0.9 err^(-1/5) taken down to the grid 2^(j/4),
// j = floor(4 log2 0.9 - 0.8 log2 err) in [-10, 13], j <= 0 after a
// rejection and j <= -1 for a rejected attempt.  The error estimate is a
// small difference of O(1) stage terms and carries rounding noise of
// relative size ~1e-16 / tol; on the grid that noise moves the step only
// when it carries the exponent across an integer, so the sequence of steps
// does not depend on rounding (and matches any other correct implementation
// of the same rule) except at those rare crossings.  Each component's
// quotient is a product with the refined reciprocal of the scale (within an
// ulp of the division, one rounding more), in the full-rate operand forms.
__device__ __forceinline__ double dopri5_norm(const BH<double>& bh, const double y[8], const double y5[8],
                                              const double e[8], double rtol, double atol) {
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double t = vmul(bh, e[q], recip<double>(fma(rtol, fmax(fabs(y[q]), fabs(y5[q])), atol), bh.one));
    s = fma(t, t, s);
  }
  return sqrt(0.125 * s);
}

__device__ __forceinline__ double dopri5_factor(double err, bool accepted, bool after_reject) {
  double q = err > 0.0 ? 4.0 * log2(0.9) - 0.8 * log2(err) : 13.0;
  const double jmax = accepted ? (after_reject ? 0.0 : 13.0) : -1.0;
  q = fmax(fmin(q, jmax), -10.0);
  const int j = (int)floor(q);
  const int r = j & 3;          // j mod 4
  const int e = (j - r) / 4;    // floor(j / 4)
  const double quarter = r == 0 ? 1.0 : (r == 1 ? 1.1892071150027210667 : (r == 2 ? 1.4142135623730950488
                                                                                    : 1.6817928305074290861));
  return ldexp(quarter, e);
}
}  // namespace malbec

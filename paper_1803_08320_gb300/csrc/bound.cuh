// bound.cuh -- device-side initial data shared by the initial-data kernels
// and the multi-job trace kernel: u = g^{-1} p, the Bardeen prograde ISCO and
// circular orbits, SplitMix64 counters, the Kerr radial potential and the
// generic bound-orbit solve and sampler (not in the paper; see ic.cu).
#pragma once
#include <math.h>
#include <stdint.h>

namespace malbec {

constexpr double kHalfPi = 1.5707963267948966;  // fl(pi/2)
constexpr double kPi = 3.141592653589793;

// u = g^{-1} p at (r, theta) for the Kerr metric, p = (p_t, p_r, p_th, p_ph).
__device__ __forceinline__ void raise_momenta(double M, double a, double r, double th, const double p[4], double u[4]) {
  double s, c;
  sincos(th, &s, &c);
  const double a2 = a * a, s2 = s * s;
  const double rho2 = fma(a2, c * c, r * r);
  const double Delta = fma(r, r - 2.0 * M, a2);
  const double q = 2.0 * M * r / rho2;
  const double gtt = q - 1.0;
  const double gtp = -a * s2 * q;
  const double gpp = s2 * fma(a2 * s2, q, r * r + a2);
  const double det = -Delta * s2;  // g_tt g_phph - g_tph^2
  u[0] = (gpp * p[0] - gtp * p[3]) / det;
  u[1] = Delta / rho2 * p[1];
  u[2] = p[2] / rho2;
  u[3] = (gtt * p[3] - gtp * p[0]) / det;
}

__device__ __forceinline__ double isco_prograde(double M, double a) {
  const double x = a / M;
  const double z1 = 1.0 + cbrt(1.0 - x * x) * (cbrt(1.0 + x) + cbrt(1.0 - x));
  const double z2 = sqrt(3.0 * x * x + z1 * z1);
  return M * (3.0 + z2 - sqrt((3.0 - z1) * (3.0 + z1 + 2.0 * z2)));
}

// Bardeen circular orbit energy and angular momentum (sg = +1 prograde).
__device__ __forceinline__ void circular_EL(double M, double a, double r, double sg, double* E, double* L) {
  const double sr = sqrt(r), sM = sqrt(M);
  const double den = sqrt(sr) * sr * sqrt(r * sr - 3.0 * M * sr + sg * 2.0 * a * sM);  // r^{3/4} sqrt(...)
  *E = (r * sr - 2.0 * M * sr + sg * a * sM) / den;
  *L = sg * sM * (r * r - sg * 2.0 * a * sM * sr + a * a) / den;
}

// ---- SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t counter) {
  return (double)(splitmix64(seed, counter) >> 11) * 0x1.0p-53;
}

// Kerr radial potential (mu = 1) and its partial derivatives with respect to
// r, E and L (L_z = L ci, Q = L^2 si^2).
struct RadialEval {
  double R, dR_dr, dR_dE, dR_dL, dRr_dE, dRr_dL;
};
__device__ __forceinline__ RadialEval radial(double M, double a, double E, double L, double ci, double si, double r) {
  const double Lz = L * ci, Q = L * L * si * si;
  const double Delta = r * r - 2.0 * M * r + a * a;
  const double P = E * (r * r + a * a) - a * Lz;
  const double B = Lz - a * E;
  const double K = r * r + B * B + Q;
  RadialEval o;
  o.R = P * P - Delta * K;
  o.dR_dr = 4.0 * E * r * P - (2.0 * r - 2.0 * M) * K - 2.0 * r * Delta;
  // d/dE and d/dL of R
  o.dR_dE = 2.0 * P * (r * r + a * a) + 2.0 * a * Delta * B;
  o.dR_dL = -2.0 * a * ci * P - Delta * (2.0 * B * ci + 2.0 * L * si * si);
  // d/dE and d/dL of R'(r)
  o.dRr_dE = 4.0 * r * P + 4.0 * E * r * (r * r + a * a) + (2.0 * r - 2.0 * M) * 2.0 * a * B;
  o.dRr_dL = -4.0 * E * r * a * ci - (2.0 * r - 2.0 * M) * (2.0 * B * ci + 2.0 * L * si * si);
  return o;
}

// Bound-orbit solve; returns 0 when the candidate is bound and stable.
__device__ inline int bound_solve(double M, double a, double rp, double e, double iota, double* E_out, double* Lz_out,
                           double* Q_out) {
  const bool circ = e < 1e-6;
  const double ra = circ ? rp : rp * (1.0 + e) / (1.0 - e);
  double si, ci;
  sincos(iota, &si, &ci);
  const double pM = rp * (1.0 + e) / M;
  const double den = pM - 3.0 - e * e;
  double E, L;
  if (den > 0.05) {
    E = sqrt((pM - 2.0 - 2.0 * e) * (pM - 2.0 + 2.0 * e) / (pM * den));
    L = M * pM / sqrt(den);
  } else {
    E = 0.95;
    L = 4.0 * M;
  }
  const double scale = rp * rp * rp * rp;
  bool ok = false;
  for (int it = 0; it < 200; ++it) {
    const RadialEval f1 = radial(M, a, E, L, ci, si, rp);
    const RadialEval f2 = radial(M, a, E, L, ci, si, ra);
    const double F0 = f1.R;
    const double F1 = circ ? f1.dR_dr : f2.R;
    if (fabs(F0) < 1e-14 * scale && fabs(F1) < 1e-14 * scale) {
      ok = true;
      break;
    }
    const double J00 = f1.dR_dE, J01 = f1.dR_dL;
    const double J10 = circ ? f1.dRr_dE : f2.dR_dE;
    const double J11 = circ ? f1.dRr_dL : f2.dR_dL;
    const double det = J00 * J11 - J01 * J10;
    if (det == 0.0 || !isfinite(det)) break;
    const double sE = -(J11 * F0 - J01 * F1) / det;
    const double sL = -(-J10 * F0 + J00 * F1) / det;
    double fac = 1.0;
    if (fabs(sE) > 0.1 * fabs(E)) fac = fmin(fac, 0.1 * fabs(E) / fabs(sE));
    if (fabs(sL) > 0.1 * fabs(L)) fac = fmin(fac, 0.1 * fabs(L) / fabs(sL));
    E += fac * sE;
    L += fac * sL;
  }
  if (!ok) {
    const RadialEval f1 = radial(M, a, E, L, ci, si, rp);
    const RadialEval f2 = radial(M, a, E, L, ci, si, ra);
    const double F1 = circ ? f1.dR_dr : f2.R;
    if (!(fabs(f1.R) < 1e-11 * scale && fabs(F1) < 1e-11 * scale)) return 1;
  }
  if (!(E > 0.0 && E < 1.0) || !(L > 0.0)) return 2;
  const double Lz = L * ci, Q = L * L * si * si;
  // remaining roots r3, r4 of R: sum 2M/(1-E^2) - ra - rp, product a^2 Q/((1-E^2) ra rp)
  const double S = 2.0 * M / (1.0 - E * E) - ra - rp;
  const double Pr = a * a * Q / ((1.0 - E * E) * ra * rp);
  const double disc = S * S - 4.0 * Pr;
  const double r3 = disc >= 0.0 ? 0.5 * (S + sqrt(disc)) : -INFINITY;
  if (r3 >= rp) return 3;
  if (!circ && !(radial(M, a, E, L, ci, si, 0.5 * (rp + ra)).R > 0.0)) return 4;
  *E_out = E;
  *Lz_out = Lz;
  *Q_out = Q;
  return 0;
}

// Seeded generic bound-orbit sample `idx` (see malbec_ic_bound): writes the
// state, returns the accepted candidate index or -1 for the fallback orbit.
__device__ inline int bound_sample(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t idx, double y[8],
                                   double* a_out) {
  const uint64_t base = idx * 256ull;
  const double a = spin_fixed ? a_max : a_max * uniform01(seed, base);
  const double r_lo = isco_prograde(M, a) + 0.5 * M, r_hi = 10.0 * M;
  int acc = -1;
  for (int j = 0; j < 64; ++j) {
    const double rp = r_lo + (r_hi - r_lo) * uniform01(seed, base + 4ull * j + 1ull);
    const double e = 0.7 * uniform01(seed, base + 4ull * j + 2ull);
    const double iota = kPi * uniform01(seed, base + 4ull * j + 3ull);
    double E, Lz, Q;
    if (bound_solve(M, a, rp, e, iota, &E, &Lz, &Q) == 0) {
      const double p[4] = {-E, 0.0, sqrt(Q), Lz};
      double u[4];
      raise_momenta(M, a, rp, kHalfPi, p, u);
      y[0] = 0.0; y[1] = rp; y[2] = kHalfPi; y[3] = 0.0;
      y[4] = u[0]; y[5] = u[1]; y[6] = u[2]; y[7] = u[3];
      acc = j;
      break;
    }
  }
  if (acc < 0) {
    double E, L;
    circular_EL(M, a, r_hi, 1.0, &E, &L);
    const double p[4] = {-E, 0.0, 0.0, L};
    double u[4];
    raise_momenta(M, a, r_hi, kHalfPi, p, u);
    y[0] = 0.0; y[1] = r_hi; y[2] = kHalfPi; y[3] = 0.0;
    y[4] = u[0]; y[5] = u[1]; y[6] = u[2]; y[7] = u[3];
  }
  *a_out = a;
  return acc;
}

}  // namespace malbec

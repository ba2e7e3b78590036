/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * What it computes, and where each piece comes from (Quiroga, arXiv:1803.08320):
 *   - the Kerr metric in Boyer-Lindquist coordinates with rho^2, Delta, Sigma
 *     (Sec. 2, eq. kerr) and its ADM lapse/shift/3-metric (Sec. 2, after eq. coord);
 *   - the geodesic equation; the paper integrates the canonical form (Sec. 2,
 *     eq. Ham); the oracle integrates the equivalent second-order form
 *     d2x/dl2 = -Gamma u u with Gamma built generically from analytic metric
 *     derivatives in plain 4x4x4 loops (form 0), and the canonical equations
 *     themselves with g of eq. kerr (form 1) or with g assembled from the
 *     lapse, shift and 3-metric of eq. ADM (form 2);
 *   - classical RK4 (Sec. 5 names the classical fourth-order method without
 *     printing its tableau: c = (0, 1/2, 1/2, 1), b = (1, 2, 2, 1)/6), and,
 *     as method 1, the Dormand-Prince 5(4) pair with step-size control (the
 *     paper's conclusions name further Runge-Kutta methods) [not in paper];
 *   - the per-ray horizon stop (Sec. 5), generalised to r <= (1+eps) r_+, plus
 *     escape r >= r_esc, a non-finite check and a step cap;
 *   - circular equatorial orbits: Schwarzschild eqs. COrbit, COrbit2,
 *     gralorbits (Sec. 4); Kerr eqs. energia, momento (Sec. 3) and Bardeen's
 *     closed forms; ISCO (eq. ISCO, eq. iscokerr, Bardeen-Press-Teukolsky);
 *     angular frequency eq. omega;
 *   - textbook additions the paper does not contain, each marked [not in paper]:
 *     Carter constant, photon-orbit radii, the backward camera, the generic
 *     bound-orbit solve and the SplitMix64 counter-based generator.
 * Compile with -O2 -fno-fast-math -ffp-contract=off so that x86 and Arm hosts
 * round identically.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX2(m, n) ((m) * 4 + (n))
#define IDX3(s, m, n) ((s) * 16 + (m) * 4 + (n))

/* ------------------------------------------------------------------------ */
/* geometry                                                                  */
/* ------------------------------------------------------------------------ */

/* Outer horizon r_+ = M + sqrt(M^2 - a^2) (Sec. 3, text after eq. ISCO). */
double orc_r_plus(double M, double a) { return M + sqrt(M * M - a * a); }

/* Kerr line element in BL coordinates, Sec. 2 eq. kerr:
 *   g_tt = -(Delta - a^2 sin^2)/rho^2, g_tphi = -2 a M r sin^2/rho^2,
 *   g_rr = rho^2/Delta, g_thth = rho^2, g_phph = Sigma sin^2/rho^2. */
void orc_metric(double M, double a, double r, double th, double g[16]) {
  double s = sin(th), c = cos(th);
  double rho2 = r * r + a * a * c * c;
  double Delta = r * r - 2.0 * M * r + a * a;
  double Sigma = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s * s;
  memset(g, 0, 16 * sizeof(double));
  g[IDX2(0, 0)] = -(Delta - a * a * s * s) / rho2;
  g[IDX2(0, 3)] = -2.0 * a * M * r * s * s / rho2;
  g[IDX2(3, 0)] = g[IDX2(0, 3)];
  g[IDX2(1, 1)] = rho2 / Delta;
  g[IDX2(2, 2)] = rho2;
  g[IDX2(3, 3)] = Sigma * s * s / rho2;
}

/* Analytic partial derivatives of the components above (only d/dr and d/dtheta
 * are non-zero: the metric does not depend on t or phi).  Each component is a
 * quotient N/D; the quotient rule is applied to the numerators and
 * denominators exactly as written in eq. kerr. */
void orc_metric_derivs(double M, double a, double r, double th, double dg[64]) {
  double s = sin(th), c = cos(th);
  double rho2 = r * r + a * a * c * c;
  double Delta = r * r - 2.0 * M * r + a * a;
  double Sigma = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s * s;
  /* derivatives of the building blocks; index 0 -> d/dr, 1 -> d/dtheta */
  double drho2[2] = {2.0 * r, -2.0 * a * a * s * c};
  double dDelta[2] = {2.0 * r - 2.0 * M, 0.0};
  double dSigma[2] = {4.0 * r * (r * r + a * a) - a * a * dDelta[0] * s * s,
                      -a * a * Delta * 2.0 * s * c};
  double ds2[2] = {0.0, 2.0 * s * c};
  memset(dg, 0, 64 * sizeof(double));
  for (int k = 0; k < 2; ++k) {
    int sidx = k + 1; /* coordinate index: r = 1, theta = 2 */
    /* g_tt = -Ntt/rho2, Ntt = Delta - a^2 s^2 */
    double Ntt = Delta - a * a * s * s;
    double dNtt = dDelta[k] - a * a * ds2[k];
    dg[IDX3(sidx, 0, 0)] = -(dNtt * rho2 - Ntt * drho2[k]) / (rho2 * rho2);
    /* g_tphi = Ntp/rho2, Ntp = -2 a M r s^2 */
    double Ntp = -2.0 * a * M * r * s * s;
    double dNtp = (k == 0) ? -2.0 * a * M * s * s : -2.0 * a * M * r * ds2[1];
    dg[IDX3(sidx, 0, 3)] = (dNtp * rho2 - Ntp * drho2[k]) / (rho2 * rho2);
    dg[IDX3(sidx, 3, 0)] = dg[IDX3(sidx, 0, 3)];
    /* g_rr = rho2/Delta */
    dg[IDX3(sidx, 1, 1)] = (drho2[k] * Delta - rho2 * dDelta[k]) / (Delta * Delta);
    /* g_thth = rho2 */
    dg[IDX3(sidx, 2, 2)] = drho2[k];
    /* g_phph = Npp/rho2, Npp = Sigma s^2 */
    double Npp = Sigma * s * s;
    double dNpp = dSigma[k] * s * s + Sigma * ds2[k];
    dg[IDX3(sidx, 3, 3)] = (dNpp * rho2 - Npp * drho2[k]) / (rho2 * rho2);
  }
}

/* Inverse metric: closed-form inverse of the (t, phi) block, reciprocal of the
 * diagonal (r, theta) entries. */
void orc_inverse_metric(double M, double a, double r, double th, double gi[16]) {
  double g[16];
  orc_metric(M, a, r, th, g);
  double det = g[IDX2(0, 0)] * g[IDX2(3, 3)] - g[IDX2(0, 3)] * g[IDX2(0, 3)];
  memset(gi, 0, 16 * sizeof(double));
  gi[IDX2(0, 0)] = g[IDX2(3, 3)] / det;
  gi[IDX2(0, 3)] = -g[IDX2(0, 3)] / det;
  gi[IDX2(3, 0)] = gi[IDX2(0, 3)];
  gi[IDX2(3, 3)] = g[IDX2(0, 0)] / det;
  gi[IDX2(1, 1)] = 1.0 / g[IDX2(1, 1)];
  gi[IDX2(2, 2)] = 1.0 / g[IDX2(2, 2)];
}

/* Christoffel symbols of the second kind, generic definition:
 *   Gamma^m_{ab} = 1/2 g^{mn} (d_a g_{nb} + d_b g_{na} - d_n g_{ab}).
 * G[m*16 + a*4 + b]. */
void orc_christoffel(double M, double a, double r, double th, double G[64]) {
  double gi[16], dg[64];
  orc_inverse_metric(M, a, r, th, gi);
  orc_metric_derivs(M, a, r, th, dg);
  for (int m = 0; m < 4; ++m)
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) {
        double sum = 0.0;
        for (int n = 0; n < 4; ++n)
          sum += gi[IDX2(m, n)] *
                 (dg[IDX3(al, n, be)] + dg[IDX3(be, n, al)] - dg[IDX3(n, al, be)]);
        G[IDX3(m, al, be)] = 0.5 * sum;
      }
}

/* ADM quantities of Kerr (Sec. 2, the comparison of eq. ADM with eq. kerr):
 * alpha = sqrt(rho^2 Delta / Sigma), beta^phi = -2 M a r / Sigma,
 * gamma = diag(rho^2/Delta, rho^2, Sigma sin^2/rho^2). */
void orc_adm(double M, double a, double r, double th, double* alpha, double* beta_phi,
             double gamma[3]) {
  double s = sin(th), c = cos(th);
  double rho2 = r * r + a * a * c * c;
  double Delta = r * r - 2.0 * M * r + a * a;
  double Sigma = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s * s;
  *alpha = sqrt(rho2 * Delta / Sigma);
  *beta_phi = -2.0 * M * a * r / Sigma;
  gamma[0] = rho2 / Delta;
  gamma[1] = rho2;
  gamma[2] = Sigma * s * s / rho2;
}

/* Partial derivatives of the ADM quantities of Kerr along r (k = 0) and
 * theta (k = 1), by the chain and quotient rules on the expressions of
 * orc_adm.  dgamma[i * 2 + k] = d gamma_ii / d x^k for i = rr, thth, phph. */
void orc_adm_derivs(double M, double a, double r, double th, double dalpha[2], double dbeta_phi[2],
                    double dgamma[6]) {
  double s = sin(th), c = cos(th);
  double rho2 = r * r + a * a * c * c;
  double Delta = r * r - 2.0 * M * r + a * a;
  double Sigma = (r * r + a * a) * (r * r + a * a) - a * a * Delta * s * s;
  double alpha = sqrt(rho2 * Delta / Sigma);
  double drho2[2] = {2.0 * r, -2.0 * a * a * s * c};
  double dDelta[2] = {2.0 * r - 2.0 * M, 0.0};
  double dSigma[2] = {4.0 * r * (r * r + a * a) - a * a * dDelta[0] * s * s,
                      -a * a * Delta * 2.0 * s * c};
  double ds2[2] = {0.0, 2.0 * s * c};
  double dr[2] = {1.0, 0.0};
  for (int k = 0; k < 2; ++k) {
    /* alpha^2 = N / Sigma with N = rho^2 Delta; d alpha = d(alpha^2) / (2 alpha) */
    double N = rho2 * Delta, dN = drho2[k] * Delta + rho2 * dDelta[k];
    double dalpha2 = (dN * Sigma - N * dSigma[k]) / (Sigma * Sigma);
    dalpha[k] = dalpha2 / (2.0 * alpha);
    /* beta^phi = -2 M a r / Sigma */
    dbeta_phi[k] = (-2.0 * M * a * dr[k] * Sigma + 2.0 * M * a * r * dSigma[k]) / (Sigma * Sigma);
    /* gamma_rr = rho^2 / Delta, gamma_thth = rho^2, gamma_phph = Sigma s^2 / rho^2 */
    dgamma[0 * 2 + k] = (drho2[k] * Delta - rho2 * dDelta[k]) / (Delta * Delta);
    dgamma[1 * 2 + k] = drho2[k];
    dgamma[2 * 2 + k] = ((dSigma[k] * s * s + Sigma * ds2[k]) * rho2 - Sigma * s * s * drho2[k]) / (rho2 * rho2);
  }
}

/* The 4-metric of the line element eq. ADM, for any lapse alpha, shift
 * beta^i and spatial metric gamma_ij (gam row-major 3x3, spatial index
 * i = 0, 1, 2 for x^1, x^2, x^3):
 *   g_tt = -alpha^2 + gamma_ij beta^i beta^j,  g_ti = gamma_ij beta^j,
 *   g_ij = gamma_ij. */
static void adm_metric(double alpha, const double beta[3], const double gam[9], double g[16]) {
  double bb = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) bb += gam[i * 3 + j] * beta[i] * beta[j];
  g[IDX2(0, 0)] = -alpha * alpha + bb;
  for (int i = 0; i < 3; ++i) {
    double bi = 0.0;
    for (int j = 0; j < 3; ++j) bi += gam[i * 3 + j] * beta[j];
    g[IDX2(0, i + 1)] = bi;
    g[IDX2(i + 1, 0)] = bi;
    for (int j = 0; j < 3; ++j) g[IDX2(i + 1, j + 1)] = gam[i * 3 + j];
  }
}

/* Its derivative along one coordinate, by the product rule on adm_metric. */
static void adm_metric_deriv(double alpha, double dalpha, const double beta[3], const double dbeta[3],
                             const double gam[9], const double dgam[9], double dg[16]) {
  double dbb = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      dbb += dgam[i * 3 + j] * beta[i] * beta[j] + gam[i * 3 + j] * dbeta[i] * beta[j] +
             gam[i * 3 + j] * beta[i] * dbeta[j];
  dg[IDX2(0, 0)] = -2.0 * alpha * dalpha + dbb;
  for (int i = 0; i < 3; ++i) {
    double dbi = 0.0;
    for (int j = 0; j < 3; ++j) dbi += dgam[i * 3 + j] * beta[j] + gam[i * 3 + j] * dbeta[j];
    dg[IDX2(0, i + 1)] = dbi;
    dg[IDX2(i + 1, 0)] = dbi;
    for (int j = 0; j < 3; ++j) dg[IDX2(i + 1, j + 1)] = dgam[i * 3 + j];
  }
}

/* Kerr's lapse, shift and 3-metric (orc_adm, orc_adm_derivs) as full 3-vectors
 * and 3x3 matrices, with their derivatives along all four coordinates
 * (d/dt and d/dphi vanish: the metric is stationary and axisymmetric). */
static void kerr_adm_full(double M, double a, double r, double th, double* alpha, double dalpha[4],
                          double beta[3], double dbeta[12], double gam[9], double dgam[36]) {
  double bphi, gd[3], da[2], db[2], dgd[6];
  orc_adm(M, a, r, th, alpha, &bphi, gd);
  orc_adm_derivs(M, a, r, th, da, db, dgd);
  memset(dalpha, 0, 4 * sizeof(double));
  memset(beta, 0, 3 * sizeof(double));
  memset(dbeta, 0, 12 * sizeof(double));
  memset(gam, 0, 9 * sizeof(double));
  memset(dgam, 0, 36 * sizeof(double));
  beta[2] = bphi;
  for (int i = 0; i < 3; ++i) gam[i * 3 + i] = gd[i];
  for (int k = 0; k < 2; ++k) {
    int s = k + 1; /* coordinate index: r = 1, theta = 2 */
    dalpha[s] = da[k];
    dbeta[s * 3 + 2] = db[k];
    for (int i = 0; i < 3; ++i) dgam[s * 9 + i * 3 + i] = dgd[i * 2 + k];
  }
}

/* Kerr's 4-metric and its derivatives assembled from the ADM quantities
 * (a different route to orc_metric and orc_metric_derivs). */
void orc_adm_metric(double M, double a, double r, double th, double g[16]) {
  double alpha, dalpha[4], beta[3], dbeta[12], gam[9], dgam[36];
  kerr_adm_full(M, a, r, th, &alpha, dalpha, beta, dbeta, gam, dgam);
  adm_metric(alpha, beta, gam, g);
}

void orc_adm_metric_derivs(double M, double a, double r, double th, double dg[64]) {
  double alpha, dalpha[4], beta[3], dbeta[12], gam[9], dgam[36];
  kerr_adm_full(M, a, r, th, &alpha, dalpha, beta, dbeta, gam, dgam);
  for (int s = 0; s < 4; ++s)
    adm_metric_deriv(alpha, dalpha[s], beta, dbeta + s * 3, gam, dgam + s * 9, dg + s * 16);
}

/* Inverse of a 4x4 matrix by Gauss-Jordan elimination with partial pivoting. */
void orc_invert4(const double A[16], double Ai[16]) {
  double w[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      w[i][j] = A[IDX2(i, j)];
      w[i][4 + j] = (i == j) ? 1.0 : 0.0;
    }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int i = col + 1; i < 4; ++i)
      if (fabs(w[i][col]) > fabs(w[piv][col])) piv = i;
    if (piv != col)
      for (int j = 0; j < 8; ++j) {
        double t = w[col][j];
        w[col][j] = w[piv][j];
        w[piv][j] = t;
      }
    double d = w[col][col];
    for (int j = 0; j < 8; ++j) w[col][j] /= d;
    for (int i = 0; i < 4; ++i) {
      if (i == col) continue;
      double f = w[i][col];
      for (int j = 0; j < 8; ++j) w[i][j] -= f * w[col][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Ai[IDX2(i, j)] = w[i][4 + j];
}

/* ------------------------------------------------------------------------ */
/* equations of motion                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  double M, a;
} orc_bh;

/* dx^m/dl = u^m, du^m/dl = -Gamma^m_{ab} u^a u^b (full 4x4 double sum). */
void orc_rhs(double M, double a, const double y[8], double f[8]) {
  double G[64];
  orc_christoffel(M, a, y[1], y[2], G);
  for (int m = 0; m < 4; ++m) {
    f[m] = y[4 + m];
    double acc = 0.0;
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) acc += G[IDX3(m, al, be)] * y[4 + al] * y[4 + be];
    f[4 + m] = -acc;
  }
}

/* Canonical equations, Sec. 2 eq. Ham with H = 1/2 g^{mn} p_m p_n:
 *   dx^m/dl = g^{mn} p_n,  dp_m/dl = -1/2 (d_m g^{ab}) p_a p_b,
 * where d_s g^{ab} = -g^{am} (d_s g_{mn}) g^{nb}. */
void orc_rhs_hamiltonian(double M, double a, const double z[8], double f[8]) {
  double gi[16], dg[64];
  orc_inverse_metric(M, a, z[1], z[2], gi);
  orc_metric_derivs(M, a, z[1], z[2], dg);
  for (int m = 0; m < 4; ++m) {
    double acc = 0.0;
    for (int n = 0; n < 4; ++n) acc += gi[IDX2(m, n)] * z[4 + n];
    f[m] = acc;
  }
  for (int s = 0; s < 4; ++s) {
    double acc = 0.0;
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) {
        double dgi = 0.0;
        for (int m = 0; m < 4; ++m)
          for (int n = 0; n < 4; ++n) dgi -= gi[IDX2(al, m)] * dg[IDX3(s, m, n)] * gi[IDX2(n, be)];
        acc += dgi * z[4 + al] * z[4 + be];
      }
    f[4 + s] = -0.5 * acc;
  }
}

/* The canonical equations (Sec. 2, eq. Ham) with the metric of the 3+1 line
 * element eq. ADM: g_{mn} and d_s g_{mn} are assembled from Kerr's lapse,
 * shift and 3-metric and their derivatives (orc_adm, orc_adm_derivs), g^{mn}
 * is their numerical 4x4 inverse; then, as in orc_rhs_hamiltonian,
 *   dx^m/dl = g^{mn} p_n,  dp_s/dl = 1/2 g^{am} (d_s g_{mn}) g^{nb} p_a p_b. */
void orc_rhs_adm(double M, double a, const double z[8], double f[8]) {
  double alpha, dalpha[4], beta[3], dbeta[12], gam[9], dgam[36];
  double g[16], gi[16];
  kerr_adm_full(M, a, z[1], z[2], &alpha, dalpha, beta, dbeta, gam, dgam);
  adm_metric(alpha, beta, gam, g);
  orc_invert4(g, gi);
  for (int m = 0; m < 4; ++m) {
    double acc = 0.0;
    for (int n = 0; n < 4; ++n) acc += gi[IDX2(m, n)] * z[4 + n];
    f[m] = acc;
  }
  for (int s = 0; s < 4; ++s) {
    double dg[16];
    adm_metric_deriv(alpha, dalpha[s], beta, dbeta + s * 3, gam, dgam + s * 9, dg);
    double acc = 0.0;
    for (int al = 0; al < 4; ++al)
      for (int be = 0; be < 4; ++be) {
        double dgi = 0.0;
        for (int m = 0; m < 4; ++m)
          for (int n = 0; n < 4; ++n) dgi -= gi[IDX2(al, m)] * dg[IDX2(m, n)] * gi[IDX2(n, be)];
        acc += dgi * z[4 + al] * z[4 + be];
      }
    f[4 + s] = -0.5 * acc;
  }
}

/* H = 1/2 g^{mn} p_m p_n with g from eq. ADM (a test handle: its finite
 * differences must reproduce orc_rhs_adm). */
double orc_hamiltonian_adm(double M, double a, const double z[8]) {
  double g[16], gi[16];
  orc_adm_metric(M, a, z[1], z[2], g);
  orc_invert4(g, gi);
  double H = 0.0;
  for (int m = 0; m < 4; ++m)
    for (int n = 0; n < 4; ++n) H += 0.5 * gi[IDX2(m, n)] * z[4 + m] * z[4 + n];
  return H;
}

typedef void (*orc_rhs_fn)(const void* ctx, const double* y, double* f);

/* One classical RK4 step of size h on a dim-dimensional system.  If
 * stage_min is given, it receives the smallest component `watch` among the
 * three intermediate stage states (the points where k2, k3, k4 are taken). */
static void rk4_generic(orc_rhs_fn fn, const void* ctx, int dim, double h, double* y, int watch,
                        double* stage_min) {
  double k1[8], k2[8], k3[8], k4[8], tmp[8];
  double mn = INFINITY;
  fn(ctx, y, k1);
  for (int i = 0; i < dim; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
  if (stage_min && tmp[watch] < mn) mn = tmp[watch];
  fn(ctx, tmp, k2);
  for (int i = 0; i < dim; ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
  if (stage_min && tmp[watch] < mn) mn = tmp[watch];
  fn(ctx, tmp, k3);
  for (int i = 0; i < dim; ++i) tmp[i] = y[i] + h * k3[i];
  if (stage_min && tmp[watch] < mn) mn = tmp[watch];
  fn(ctx, tmp, k4);
  for (int i = 0; i < dim; ++i) y[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
  if (stage_min) *stage_min = mn;
}

static void geo_fn(const void* ctx, const double* y, double* f) {
  const orc_bh* bh = (const orc_bh*)ctx;
  orc_rhs(bh->M, bh->a, y, f);
}
static void ham_fn(const void* ctx, const double* y, double* f) {
  const orc_bh* bh = (const orc_bh*)ctx;
  orc_rhs_hamiltonian(bh->M, bh->a, y, f);
}
static void adm_fn(const void* ctx, const double* y, double* f) {
  const orc_bh* bh = (const orc_bh*)ctx;
  orc_rhs_adm(bh->M, bh->a, y, f);
}
static void lin_fn(const void* ctx, const double* y, double* f) { f[0] = *(const double*)ctx * y[0]; }

void orc_rk4_linear_test(double lam, double h, int nsteps, double* y) {
  for (int i = 0; i < nsteps; ++i) rk4_generic(lin_fn, &lam, 1, h, y, 0, NULL);
}
void orc_rk4_step(double M, double a, double h, double y[8]) {
  orc_bh bh = {M, a};
  rk4_generic(geo_fn, &bh, 8, h, y, 1, NULL);
}
void orc_rk4_step_hamiltonian(double M, double a, double h, double z[8]) {
  orc_bh bh = {M, a};
  rk4_generic(ham_fn, &bh, 8, h, z, 1, NULL);
}
void orc_rk4_step_adm(double M, double a, double h, double z[8]) {
  orc_bh bh = {M, a};
  rk4_generic(adm_fn, &bh, 8, h, z, 1, NULL);
}

/* ------------------------------------------------------------------------ */
/* Dormand-Prince 5(4) (the paper's future work names more Runge-Kutta       */
/* methods, Sec. 7) [not in paper]                                            */
/* ------------------------------------------------------------------------ */

/* The coefficients of Dormand & Prince, "A family of embedded Runge-Kutta
 * formulae", J. Comput. Appl. Math. 6 (1980) 19-26: seven stages, the last
 * evaluated at the fifth-order result (a_7j = b_j), so it is the first stage
 * of the next step. */
static const double DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double DP_A[7][7] = {
    {0, 0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0}};
static const double DP_B[7] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0};
static const double DP_BH[7] = {5179.0 / 57600.0, 0.0,          7571.0 / 16695.0, 393.0 / 640.0,
                                -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

void orc_dopri5_tableau(double c[7], double a[49], double b[7], double bhat[7]) {
  for (int i = 0; i < 7; ++i) {
    c[i] = DP_C[i];
    b[i] = DP_B[i];
    bhat[i] = DP_BH[i];
    for (int j = 0; j < 7; ++j) a[i * 7 + j] = DP_A[i][j];
  }
}

/* One attempt of size h from y with k1 = f(y): the stage points
 * y_i = y + h sum_j a_ij k_j and k_i = f(y_i) for i = 2..7, the fifth-order
 * result y5 = y_7, the error estimate e = h sum_j (b_j - bhat_j) k_j, k7 =
 * f(y5), and the smallest component `watch` among the stage points 2..7. */
static void dopri5_attempt(orc_rhs_fn fn, const void* ctx, int dim, double h, const double* y,
                           const double* k1, double* y5, double* e, double* k7, int watch, double* stage_min) {
  double k[7][8], ys[8];
  double mn = INFINITY;
  for (int q = 0; q < dim; ++q) k[0][q] = k1[q];
  for (int i = 1; i < 7; ++i) {
    for (int q = 0; q < dim; ++q) {
      double acc = 0.0;
      for (int j = 0; j < i; ++j) acc += DP_A[i][j] * k[j][q];
      ys[q] = y[q] + h * acc;
    }
    if (ys[watch] < mn) mn = ys[watch];
    fn(ctx, ys, k[i]);
  }
  for (int q = 0; q < dim; ++q) {
    y5[q] = ys[q];
    k7[q] = k[6][q];
    double acc = 0.0;
    for (int j = 0; j < 7; ++j) acc += (DP_B[j] - DP_BH[j]) * k[j][q];
    e[q] = h * acc;
  }
  if (stage_min) *stage_min = mn;
}

/* Root-mean-square error norm with the mixed scale atol + rtol max(|y|, |y5|)
 * (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4). */
static double dopri5_norm(int dim, const double* y, const double* y5, const double* e, double rtol, double atol) {
  double s = 0.0;
  for (int q = 0; q < dim; ++q) {
    double sc = atol + rtol * fmax(fabs(y[q]), fabs(y5[q]));
    s += (e[q] / sc) * (e[q] / sc);
  }
  return sqrt(s / dim);
}

/* Step-size factor after an attempt with error norm err: the usual
 * 0.9 err^(-1/5) (safety 0.9, exponent 1/5 for the fifth-order pair) taken
 * down to the grid 2^(j/4), j = floor(4 log2 0.9 - 0.8 log2 err), with j in
 * [-10, 13] (factors 0.18 .. 9.5), j <= 0 for the step after a rejection and
 * j <= -1 after a rejection itself.  The embedded error estimate is a small
 * difference of O(1) terms, so err carries rounding noise of relative size
 * ~1e-16 / tol; on the grid that noise changes the step only when it moves
 * the exponent across an integer, and the sequence of steps is the same for
 * any two correct implementations (a continuous factor would pass the noise
 * into every step and end a fixed number of attempts at a slightly
 * different lambda) [not in paper]. */
static double dopri5_factor(double err, int accepted, int after_reject) {
  double q = err > 0.0 ? 4.0 * log2(0.9) - 0.8 * log2(err) : 13.0;
  int jmax = accepted ? (after_reject ? 0 : 13) : -1;
  if (q > (double)jmax) q = (double)jmax;
  if (q < -10.0) q = -10.0;
  int j = (int)floor(q);
  int r = j & 3;        /* j mod 4, in 0..3 */
  int e = (j - r) / 4;  /* floor(j / 4) */
  static const double quarter[4] = {1.0, 1.1892071150027210667, 1.4142135623730950488, 1.6817928305074290861};
  return ldexp(quarter[r], e);
}

void orc_dopri5_linear_test(double lam, double h, double y0, double* y5, double* err) {
  double k1 = lam * y0, k7, e;
  dopri5_attempt(lin_fn, &lam, 1, h, &y0, &k1, y5, &e, &k7, 0, NULL);
  *err = e;
}

/* ------------------------------------------------------------------------ */
/* integration with termination                                              */
/* ------------------------------------------------------------------------ */

static int all_finite(const double y[8]) {
  for (int i = 0; i < 8; ++i)
    if (!isfinite(y[i])) return 0;
  return 1;
}

/* Integrate one ray.  After every completed step: captured if the radius
 * reached (1+eps) r_+ (the paper's per-thread horizon stop, Sec. 5) -- at the
 * new state or at any of the step's intermediate stage points, since a stage
 * that lands inside r_+ (Delta < 0) spoils the whole step; else non-finite if
 * any component is not finite; else escaped if r >= r_esc; after n_steps_cap
 * steps: capped.  The reported state is the post-step state.  The step size
 * is fixed (dl) or dl_r_scale * r at the start of the step, held for all four
 * stages.  traj (optional) receives sample k (k*stride steps) at
 * traj[k*8 ...]; samples after termination are NaN. */
/* (x, p) -> (x, u): u^m = g^{mn} p_n, with g^{mn} of eq. kerr (form 1) or the
 * inverse of the eq. ADM metric (form 2). */
static void canonical_to_state(double M, double a, int form, const double z[8], double y[8]) {
  double gi[16];
  if (form == 2) {
    double g[16];
    orc_adm_metric(M, a, z[1], z[2], g);
    orc_invert4(g, gi);
  } else {
    orc_inverse_metric(M, a, z[1], z[2], gi);
  }
  for (int m = 0; m < 4; ++m) {
    double acc = 0.0;
    for (int n = 0; n < 4; ++n) acc += gi[IDX2(m, n)] * z[4 + n];
    y[m] = z[m];
    y[4 + m] = acc;
  }
}

/* The rhs_noise option: wrap a right-hand side so that every component of
 * every evaluation is scaled by 1 +- noise (sign from SplitMix64 seeded with
 * the bits of `noise`, on the evaluation counter and the component index). */
typedef struct {
  orc_rhs_fn fn;
  const void* ctx;
  double noise;
  uint64_t count;
} noisy_rhs;
static void noisy_fn(const void* c, const double* y, double* f) {
  noisy_rhs* n = (noisy_rhs*)c;
  n->fn(n->ctx, y, f);
  uint64_t seed;
  memcpy(&seed, &n->noise, sizeof(seed)); /* another noise value, another sign pattern */
  for (int i = 0; i < 8; ++i) {
    uint64_t b = orc_splitmix64(seed, n->count * 8u + (uint64_t)i);
    f[i] *= 1.0 + ((b >> 63) ? n->noise : -n->noise);
  }
  n->count++;
}

int orc_trace_one(double M, double a, const double y0[8], const orc_term* t, double y[8],
                  double* lambda, uint32_t* steps, double* traj, uint32_t stride) {
  double r_cap = (1.0 + t->eps_hor) * orc_r_plus(M, a);
  uint32_t ns = (traj && stride) ? t->n_steps_cap / stride + 1 : 0;
  int fate = ORC_FATE_CAPPED;
  uint32_t n = 0;
  double lam = 0.0;
  /* the integrated state: (x, u), or (x, p) with p = g u in the canonical
   * forms (1: g of eq. kerr, 2: g of eq. ADM); inputs, samples and the
   * result are (x, u) in all three */
  const int form = (int)t->form;
  const int canonical = form == 1 || form == 2;
  orc_rhs_fn rhs = form == 2 ? adm_fn : (form == 1 ? ham_fn : geo_fn);
  double z[8];
  memcpy(y, y0, 8 * sizeof(double));
  memcpy(z, y0, 8 * sizeof(double));
  if (form == 1) orc_state_to_momenta(M, a, y0, z + 4);
  if (form == 2) {
    double g[16];
    orc_adm_metric(M, a, y0[1], y0[2], g);
    for (int m = 0; m < 4; ++m) {
      z[4 + m] = 0.0;
      for (int n = 0; n < 4; ++n) z[4 + m] += g[IDX2(m, n)] * y0[4 + n];
    }
  }
  if (ns) memcpy(traj, y, 8 * sizeof(double));
  orc_bh bh = {M, a};
  const void* rctx = &bh;
  noisy_rhs noisy = {rhs, &bh, t->rhs_noise, 0u};
  if (t->rhs_noise != 0.0) {
    rhs = noisy_fn;
    rctx = &noisy;
  }
  if (t->method == 1) {
    /* Dormand-Prince 5(4) with step-size control; n counts attempts; the
     * termination tests follow every attempt (capture and non-finite on the
     * attempted state, escape on accepted states) */
    double h = t->dl > 0.0 ? t->dl : t->dl_r_scale * z[1];
    double k1[8], y5[8], e[8], k7[8];
    int after_reject = 0;
    rhs(rctx, z, k1);
    while (n < t->n_steps_cap) {
      if (t->dl_r_scale > 0.0 && h > t->dl_r_scale * z[1]) h = t->dl_r_scale * z[1];
      double r_stage_min;
      dopri5_attempt(rhs, rctx, 8, h, z, k1, y5, e, k7, 1, &r_stage_min);
      ++n;
      int done = 0;
      if (y5[1] <= r_cap || r_stage_min <= r_cap) {
        fate = ORC_FATE_CAPTURED;
        done = 1;
      } else if (!all_finite(y5)) {
        fate = ORC_FATE_NONFINITE;
        done = 1;
      }
      if (done) {
        memcpy(z, y5, 8 * sizeof(double));
        lam += h;
      } else {
        double err = dopri5_norm(8, z, y5, e, t->rtol, t->atol);
        if (err <= 1.0) {
          memcpy(z, y5, 8 * sizeof(double));
          memcpy(k1, k7, 8 * sizeof(double));
          lam += h;
          h *= dopri5_factor(err, 1, after_reject);
          after_reject = 0;
          if (z[1] >= t->r_esc) {
            fate = ORC_FATE_ESCAPED;
            done = 1;
          }
        } else {
          h *= dopri5_factor(err, 0, 0);
          after_reject = 1;
        }
      }
      if (ns && n % stride == 0) {
        double* s = traj + (size_t)(n / stride) * 8;
        if (canonical)
          canonical_to_state(M, a, form, z, s);
        else
          memcpy(s, z, 8 * sizeof(double));
      }
      if (done) break;
    }
  }
  while (t->method != 1 && n < t->n_steps_cap) {
    double h = (t->dl_r_scale > 0.0) ? t->dl_r_scale * z[1] : t->dl;
    double r_stage_min;
    rk4_generic(rhs, rctx, 8, h, z, 1, &r_stage_min);
    lam += h;
    ++n;
    if (ns && n % stride == 0) {
      double* s = traj + (size_t)(n / stride) * 8;
      if (canonical)
        canonical_to_state(M, a, form, z, s);
      else
        memcpy(s, z, 8 * sizeof(double));
    }
    if (z[1] <= r_cap || r_stage_min <= r_cap) { fate = ORC_FATE_CAPTURED; break; }
    if (!all_finite(z)) { fate = ORC_FATE_NONFINITE; break; }
    if (z[1] >= t->r_esc) { fate = ORC_FATE_ESCAPED; break; }
  }
  if (canonical)
    canonical_to_state(M, a, form, z, y);
  else
    memcpy(y, z, 8 * sizeof(double));
  if (ns)
    for (uint32_t k = n / stride + 1; k < ns; ++k)
      for (int c = 0; c < 8; ++c) traj[(size_t)k * 8 + c] = NAN;
  /* validity: the norm g(u,u) is a constant of the flow */
  if (fate == ORC_FATE_ESCAPED || fate == ORC_FATE_CAPPED) {
    double i0[4], i1[4];
    orc_invariants(M, a, y0, i0);
    orc_invariants(M, a, y, i1);
    double lim = ORC_NORM_DRIFT_TOL * fmax(i0[0] * i0[0], fabs(i0[3]));
    if (fabs(i1[3] - i0[3]) > lim) fate |= ORC_FATE_DRIFTED;
  }
  *lambda = lam;
  *steps = n;
  return fate;
}

int orc_trace_many(double M, double a, const double* a_per_ray, const double* ics, uint64_t n,
                   const orc_term* t, double* y_out, double* lambda, double* inv0, double* inv1,
                   uint32_t* steps, uint8_t* fate, double* traj, uint32_t stride, int nthreads) {
  int used = 1;
  size_t ns = (traj && stride) ? t->n_steps_cap / stride + 1 : 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  used = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t i = 0; i < (int64_t)n; ++i) {
    double ai = a_per_ray ? a_per_ray[i] : a;
    double y0[8], y[8], inv[4], lam;
    uint32_t st;
    for (int c = 0; c < 8; ++c) y0[c] = ics[(size_t)c * n + i];
    if (inv0) {
      orc_invariants(M, ai, y0, inv);
      for (int c = 0; c < 4; ++c) inv0[(size_t)c * n + i] = inv[c];
    }
    int f = orc_trace_one(M, ai, y0, t, y, &lam, &st, ns ? traj + (size_t)i * ns * 8 : NULL, stride);
    for (int c = 0; c < 8; ++c) y_out[(size_t)c * n + i] = y[c];
    if (lambda) lambda[i] = lam;
    if (steps) steps[i] = st;
    if (fate) fate[i] = (uint8_t)f;
    if (inv1) {
      orc_invariants(M, ai, y, inv);
      for (int c = 0; c < 4; ++c) inv1[(size_t)c * n + i] = inv[c];
    }
  }
  return used;
}

/* ------------------------------------------------------------------------ */
/* conserved quantities                                                      */
/* ------------------------------------------------------------------------ */

/* p_m = g_{mn} u^n; E = -p_t; L_z = p_phi; norm = g_{mn} u^m u^n (the
 * constraint 2L = -1 of eq. geo for timelike, 0 for null); Carter's constant
 * [not in paper] Q = p_th^2 + cos^2 th (a^2 (mu^2 - E^2) + L_z^2 / sin^2 th)
 * with mu^2 = -norm. */
void orc_invariants(double M, double a, const double y[8], double inv[4]) {
  double g[16], p[4];
  orc_metric(M, a, y[1], y[2], g);
  double norm = 0.0;
  for (int m = 0; m < 4; ++m) {
    p[m] = 0.0;
    for (int n = 0; n < 4; ++n) p[m] += g[IDX2(m, n)] * y[4 + n];
    norm += p[m] * y[4 + m];
  }
  double E = -p[0], Lz = p[3], mu2 = -norm;
  double s = sin(y[2]), c = cos(y[2]);
  inv[0] = E;
  inv[1] = Lz;
  inv[2] = p[2] * p[2] + c * c * (a * a * (mu2 - E * E) + Lz * Lz / (s * s));
  inv[3] = norm;
}

/* ------------------------------------------------------------------------ */
/* initial conditions                                                        */
/* ------------------------------------------------------------------------ */

static void momenta_to_state(double M, double a, const double x[4], const double p[4], double y[8]) {
  double gi[16];
  orc_inverse_metric(M, a, x[1], x[2], gi);
  for (int m = 0; m < 4; ++m) {
    y[m] = x[m];
    double acc = 0.0;
    for (int n = 0; n < 4; ++n) acc += gi[IDX2(m, n)] * p[n];
    y[4 + m] = acc;
  }
}

/* The paper's initial-condition rows (Sec. 5: t, r, th, ph, p_t, p_r, p_th,
 * p_ph) list p_t = +E; covariant p_t = -E.  u^m = g^{mn} p_n. */
void orc_paper_to_state(double M, double a, const double xp[8], double y[8]) {
  double p[4] = {-xp[4], xp[5], xp[6], xp[7]};
  momenta_to_state(M, a, xp, p, y);
}

void orc_state_to_momenta(double M, double a, const double y[8], double p[4]) {
  double g[16];
  orc_metric(M, a, y[1], y[2], g);
  for (int m = 0; m < 4; ++m) {
    p[m] = 0.0;
    for (int n = 0; n < 4; ++n) p[m] += g[IDX2(m, n)] * y[4 + n];
  }
}

/* BL -> Cartesian map, Sec. 2 eq. coord. */
void orc_bl_to_cartesian(double a, double r, double th, double ph, double xyz[3]) {
  double R = sqrt(r * r + a * a);
  xyz[0] = R * sin(th) * cos(ph);
  xyz[1] = R * sin(th) * sin(ph);
  xyz[2] = r * cos(th);
}

/* Schwarzschild circular orbits, Sec. 4 eqs. COrbit, COrbit2:
 * E^2 = (4M^2 - 4Mr + r^2)/(r(r - 3M)), L^2 = M r^2/(r - 3M). */
void orc_schw_circular(double M, double r, double* E, double* L) {
  *E = sqrt((4.0 * M * M - 4.0 * M * r + r * r) / (r * (r - 3.0 * M)));
  *L = sqrt(M * r * r / (r - 3.0 * M));
}

/* Sec. 4 eq. gralorbits with r = kM: p_t = sqrt((k^2-4k+4)/(k(k-3))), p_phi = kM/sqrt(k-3). */
void orc_schw_gralorbits(double k, double M, double* pt, double* pphi) {
  *pt = sqrt((k * k - 4.0 * k + 4.0) / (k * (k - 3.0)));
  *pphi = k * M / sqrt(k - 3.0);
}

/* Sec. 3 eqs. energia and momento exactly as printed, with the sign sgn = +1
 * or -1 taking the place of the +- symbol both inside the root and in front
 * of L; R from the definition after eq. momento. */
void orc_kerr_circular_paper(double M, double a, double r, int sgn, double* E, double* L) {
  double R = r * r *
             (-12.0 * M * M * M * r + 5.0 * M * M * a * a + 16.0 * M * M * r * r -
              3.0 * M * a * a * r - 7.0 * M * r * r * r + r * r * r * r);
  double w = 2.0 * M * r - a * a - r * r;
  double root = sqrt(R + sgn * 2.0 * pow(M, 1.5) * pow(r, 1.5) * w * a);
  *E = fabs((4.0 * M * M * r - M * a * a - 4.0 * M * r * r + r * r * r) / root);
  *L = sgn * fabs((M * a * (4.0 * M * r - a * a - 3.0 * r * r) + pow(r, 1.5) * w * sqrt(M)) / root);
}

/* Bardeen, Press & Teukolsky (1972) circular equatorial orbits [closed form,
 * the paper's reference for the ISCO limits]:
 *   E = (r^{3/2} - 2M r^{1/2} +- a M^{1/2}) / (r^{3/4} sqrt(r^{3/2} - 3M r^{1/2} +- 2a M^{1/2}))
 *   L = +- M^{1/2}(r^2 -+ 2a M^{1/2} r^{1/2} + a^2) / (same denominator)
 * upper sign prograde (co-rotating). */
void orc_kerr_circular_bardeen(double M, double a, double r, int prograde, double* E, double* L) {
  double sg = prograde ? 1.0 : -1.0;
  double sr = sqrt(r), sM = sqrt(M);
  double den = pow(r, 0.75) * sqrt(r * sr - 3.0 * M * sr + sg * 2.0 * a * sM);
  *E = (r * sr - 2.0 * M * sr + sg * a * sM) / den;
  *L = sg * sM * (r * r - sg * 2.0 * a * sM * sr + a * a) / den;
}

/* Sec. 3 eq. omega: omega = (-2 M a p_t + (2M - r) p_phi) / (r (2Mr - a^2 - r^2)),
 * with the paper's p_t = +E. */
double orc_kerr_omega(double M, double a, double r, double pt_paper, double pphi) {
  return (-2.0 * M * a * pt_paper + (2.0 * M - r) * pphi) / (r * (2.0 * M * r - a * a - r * r));
}

/* Bardeen-Press-Teukolsky ISCO:
 *   Z1 = 1 + (1 - a^2/M^2)^{1/3} ((1 + a/M)^{1/3} + (1 - a/M)^{1/3}),
 *   Z2 = sqrt(3 a^2/M^2 + Z1^2),
 *   r = M (3 + Z2 -+ sqrt((3 - Z1)(3 + Z1 + 2 Z2)))   (upper: prograde). */
double orc_isco_bardeen(double M, double a, int prograde) {
  double x = a / M;
  double Z1 = 1.0 + cbrt(1.0 - x * x) * (cbrt(1.0 + x) + cbrt(1.0 - x));
  double Z2 = sqrt(3.0 * x * x + Z1 * Z1);
  double sg = prograde ? -1.0 : 1.0;
  return M * (3.0 + Z2 + sg * sqrt((3.0 - Z1) * (3.0 + Z1 + 2.0 * Z2)));
}

/* Sec. 3 eq. iscokerr exactly as printed (sgn = +1 for the upper sign);
 * returns NaN where a square root of a negative number appears. */
double orc_isco_paper_literal(double M, double a, int sgn) {
  double a2 = a * a, M2 = M * M;
  double base = a2 * a2 * a2 + 17.0 * a2 * a2 * M2 - 45.0 * a2 * M2 * M2 + 27.0 * M2 * M2 * M2 +
                8.0 * sqrt(pow(a, 10) * M2 - 2.0 * pow(a, 8) * M2 * M2 + pow(a, 6) * M2 * M2 * M2);
  double cb = cbrt(base);
  double A = 4.0 * (a2 * a2 - 10.0 * a2 * M2 + 9.0 * M2 * M2) / cb;
  double B = 4.0 * cb;
  double C = 36.0 * M2 + 4.0 * (a2 - 6.0 * M2);
  double s1 = A + B + C;
  if (s1 < 0.0) return NAN;
  double q = -A - B + 2.0 * C + (224.0 * a2 * M + 1728.0 * M * (a2 - 6.0 * M2)) / (4.0 * sqrt(s1));
  if (q < 0.0) return NAN;
  return 3.0 * M + 0.5 * sqrt(s1) - sgn * sqrt(q);
}

/* Sec. 3 eq. ISCO: the ISCO is the root of dE/dr = 0.  dE/dr by a central
 * difference of the Bardeen E(r), root by bisection on [r_lo, r_hi]. */
static double dEdr(double M, double a, int prograde, double r) {
  double hh = 1e-5 * r, Ep, Em, L;
  orc_kerr_circular_bardeen(M, a, r + hh, prograde, &Ep, &L);
  orc_kerr_circular_bardeen(M, a, r - hh, prograde, &Em, &L);
  return (Ep - Em) / (2.0 * hh);
}
double orc_dEdr_numeric_root(double M, double a, int prograde, double r_lo, double r_hi) {
  double flo = dEdr(M, a, prograde, r_lo);
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (r_lo + r_hi);
    double fm = dEdr(M, a, prograde, mid);
    if ((fm < 0.0) == (flo < 0.0)) { r_lo = mid; flo = fm; } else { r_hi = mid; }
  }
  return 0.5 * (r_lo + r_hi);
}

/* Circular equatorial photon orbits [not in paper; Bardeen 1972]:
 * r_ph = 2M (1 + cos(2/3 arccos(-+ a/M)))  (upper: prograde). */
double orc_photon_orbit(double M, double a, int prograde) {
  double sg = prograde ? -1.0 : 1.0;
  return 2.0 * M * (1.0 + cos(2.0 / 3.0 * acos(sg * a / M)));
}

/* Circular equatorial timelike orbit at radius r: p = (-E, 0, 0, L) from the
 * Bardeen E, L; u = g^{-1} p. */
void orc_circular_state(double M, double a, double r, int prograde, double y[8]) {
  double E, L;
  orc_kerr_circular_bardeen(M, a, r, prograde, &E, &L);
  double x[4] = {0.0, r, M_PI / 2.0, 0.0};
  double p[4] = {-E, 0.0, 0.0, L};
  momenta_to_state(M, a, x, p, y);
}

/* Backward null-ray camera [not in paper; Bardeen 1973 impact parameters].
 * Pixel pix = j*nx + i, i along alpha, j along beta, pixel centres
 *   alpha = -fov + 2 fov (i + 1/2)/nx,   beta = -fov + 2 fov (j + 1/2)/ny.
 * Arriving photon: E = 1, L = -alpha sin th_o, Q = beta^2 + cos^2 th_o (alpha^2 - a^2),
 *   p_th = sign(beta) sqrt(Theta(th_o)), Theta = Q + a^2 cos^2 - L^2 cot^2,
 *   p_r = +sqrt(R(r_o))/Delta(r_o), R = ((r^2 + a^2) E - a L)^2 - Delta (Q + (L - a E)^2).
 * The ray is traced backward by integrating forward in lambda with the
 * momentum reversed, p~ = -p; u = g^{-1} p~; x = (0, r_o, th_o, 0). */
void orc_camera_ic(double M, double a, double r_o, double th_o, double fov_half, uint32_t nx,
                   uint32_t ny, uint64_t pix, double y[8]) {
  uint64_t i = pix % nx, j = pix / nx;
  double alpha = -fov_half + 2.0 * fov_half * ((double)i + 0.5) / (double)nx;
  double beta = -fov_half + 2.0 * fov_half * ((double)j + 0.5) / (double)ny;
  double E = 1.0;
  double so = sin(th_o), co = cos(th_o);
  double L = -alpha * so;
  double Q = beta * beta + co * co * (alpha * alpha - a * a);
  double Theta = Q + a * a * co * co - L * L * co * co / (so * so);
  if (Theta < 0.0) Theta = 0.0;
  double pth = (beta >= 0.0 ? 1.0 : -1.0) * sqrt(Theta);
  double Delta = r_o * r_o - 2.0 * M * r_o + a * a;
  double Rr = ((r_o * r_o + a * a) * E - a * L) * ((r_o * r_o + a * a) * E - a * L) -
              Delta * (Q + (L - a * E) * (L - a * E));
  if (Rr < 0.0) Rr = 0.0;
  double pr = sqrt(Rr) / Delta;
  double x[4] = {0.0, r_o, th_o, 0.0};
  double p[4] = {E, -pr, -pth, -L}; /* reversed: -(-E, pr, pth, L) */
  momenta_to_state(M, a, x, p, y);
}

/* The Kerr critical curve (boundary of the shadow) [not in paper; Bardeen
 * 1973], the image of the spherical photon orbits of radius r:
 *   xi(r) = (r^2 (3M - r) - a^2 (r + M)) / (a (r - M)),
 *   eta(r) = r^3 (4 a^2 M - r (r - 3M)^2) / (a^2 (r - M)^2),
 *   alpha = -xi / sin th_o, beta = +- sqrt(b2), b2 = eta + a^2 cos^2 th_o - xi^2 cot^2 th_o,
 * over the r where b2 >= 0 (the orbits whose polar range reaches th_o), a
 * sub-interval [r_a, r_b] of the photon-orbit band [r_ph,pro, r_ph,retro]; for
 * a = 0 a circle of radius 3 sqrt(3) M.  Near r_a and r_b, beta grows like
 * sqrt(r - r_a), so the curve is sampled at r = r_a + (r_b - r_a)(1 - cos(pi u))/2
 * with u uniform in [0, 1], which spaces the points evenly along beta there. */
static double cc_b2(double M, double a, double so, double co, double r, double* xi_out) {
  double xi = (r * r * (3.0 * M - r) - a * a * (r + M)) / (a * (r - M));
  double eta = r * r * r * (4.0 * a * a * M - r * (r - 3.0 * M) * (r - 3.0 * M)) / (a * a * (r - M) * (r - M));
  if (xi_out) *xi_out = xi;
  return eta + a * a * co * co - xi * xi * co * co / (so * so);
}

/* [r_a, r_b]: bisection for b2 = 0 on each side of the polar orbit
 * (xi = 0, where b2 = eta + a^2 cos^2 th_o > 0). */
static void cc_range(double M, double a, double so, double co, double* ra, double* rb) {
  double r1 = orc_photon_orbit(M, a, 1), r2 = orc_photon_orbit(M, a, 0);
  double lo = r1, hi = r2, r0;
  for (int k = 0; k < 200; ++k) { /* xi decreases from xi(r1) > 0 to xi(r2) < 0 */
    double mid = 0.5 * (lo + hi), xi;
    cc_b2(M, a, so, co, mid, &xi);
    if (xi > 0.0) lo = mid; else hi = mid;
  }
  r0 = 0.5 * (lo + hi);
  *ra = r1;
  if (cc_b2(M, a, so, co, r1, NULL) < 0.0) {
    lo = r1; hi = r0;
    for (int k = 0; k < 200; ++k) {
      double mid = 0.5 * (lo + hi);
      if (cc_b2(M, a, so, co, mid, NULL) < 0.0) lo = mid; else hi = mid;
    }
    *ra = hi;
  }
  *rb = r2;
  if (cc_b2(M, a, so, co, r2, NULL) < 0.0) {
    lo = r0; hi = r2;
    for (int k = 0; k < 200; ++k) {
      double mid = 0.5 * (lo + hi);
      if (cc_b2(M, a, so, co, mid, NULL) < 0.0) hi = mid; else lo = mid;
    }
    *rb = lo;
  }
}

/* The point of the upper branch (beta >= 0) at curve parameter u in [0, 1]. */
static void cc_point(double M, double a, double so, double co, double ra, double rb, double u,
                     double* al, double* be) {
  double r = ra + (rb - ra) * 0.5 * (1.0 - cos(M_PI * u)), xi;
  double b2 = cc_b2(M, a, so, co, r, &xi);
  *al = -xi / so;
  *be = b2 > 0.0 ? sqrt(b2) : 0.0;
}

double orc_critical_curve_distance(double M, double a, double th_o, double alpha, double beta) {
  if (fabs(a) < 1e-12) return fabs(hypot(alpha, beta) - 3.0 * sqrt(3.0) * M);
  double so = sin(th_o), co = cos(th_o), ra, rb;
  cc_range(M, fabs(a), so, co, &ra, &rb);
  double bab = fabs(beta); /* the curve is symmetric under beta -> -beta */
  int N = 20000;
  double best = INFINITY, ubest = 0.0;
  for (int k = 0; k <= N; ++k) {
    double u = (double)k / N, al, be;
    cc_point(M, fabs(a), so, co, ra, rb, u, &al, &be);
    double d = hypot(alpha - al, bab - be);
    if (d < best) { best = d; ubest = u; }
  }
  double lo = ubest - 1.0 / N, hi = ubest + 1.0 / N;
  if (lo < 0.0) lo = 0.0;
  if (hi > 1.0) hi = 1.0;
  for (int k = 0; k <= 2000; ++k) {
    double al, be;
    cc_point(M, fabs(a), so, co, ra, rb, lo + (hi - lo) * k / 2000.0, &al, &be);
    double d = hypot(alpha - al, bab - be);
    if (d < best) best = d;
  }
  return best;
}

/* The curve as a closed polyline of 2n points: the upper branch for
 * u = k/(n-1), k = 0..n-1, then the lower branch back (beta -> -beta). */
void orc_critical_curve_polyline(double M, double a, double th_o, int n, double* alpha, double* beta) {
  double so = sin(th_o), co = cos(th_o), ra = 0.0, rb = 0.0;
  if (fabs(a) >= 1e-12) cc_range(M, fabs(a), so, co, &ra, &rb);
  for (int k = 0; k < n; ++k) {
    double u = n > 1 ? (double)k / (n - 1) : 0.0, al, be;
    if (fabs(a) < 1e-12) {
      al = -3.0 * sqrt(3.0) * M * cos(M_PI * u);
      be = 3.0 * sqrt(3.0) * M * sin(M_PI * u);
    } else {
      cc_point(M, fabs(a), so, co, ra, rb, u, &al, &be);
    }
    alpha[k] = al;
    beta[k] = be;
    alpha[2 * n - 1 - k] = al;
    beta[2 * n - 1 - k] = -be;
  }
}

/* ------------------------------------------------------------------------ */
/* generic bound orbits [not in paper]                                       */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based generator:
 * the output for counter k is the SplitMix64 output after k+1 increments of
 * the state seeded with `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
/* uniform in [0, 1): top 53 bits times 2^-53 */
double orc_uniform(uint64_t seed, uint64_t counter) {
  return (double)(orc_splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

/* Kerr radial potential with mu = 1:
 * R(r) = (E (r^2 + a^2) - a L_z)^2 - Delta (r^2 + (L_z - a E)^2 + Q). */
double orc_radial_potential(double M, double a, double E, double Lz, double Q, double r) {
  double Delta = r * r - 2.0 * M * r + a * a;
  double P = E * (r * r + a * a) - a * Lz;
  return P * P - Delta * (r * r + (Lz - a * E) * (Lz - a * E) + Q);
}

/* Solve for (E, L_z, Q) of the bound orbit with periapsis rp, eccentricity e
 * (apoapsis ra = rp (1+e)/(1-e)) and inclination iota (cos iota = L_z /
 * sqrt(L_z^2 + Q)).  Unknowns (E, L) with L_z = L cos iota, Q = L^2 sin^2 iota.
 * Equations R(rp) = R(ra) = 0, or R(rp) = R'(rp) = 0 when e < 1e-6.  Newton's
 * method with a finite-difference Jacobian, from the Schwarzschild guess with
 * semi-latus rectum p = rp (1 + e).  Returns 0 for a bound, stable orbit;
 * 1 no convergence, 2 E >= 1 or E <= 0, 3 third root r3 >= rp (plunging),
 * 4 the region between rp and ra is not allowed. */
static void bound_residual(double M, double a, double rp, double ra, int circ, double ci,
                           double si, double E, double L, double F[2]) {
  double Lz = L * ci, Q = L * L * si * si;
  F[0] = orc_radial_potential(M, a, E, Lz, Q, rp);
  if (circ) {
    /* R'(r) = 2 P (2 E r) - (2r - 2M)(r^2 + (L_z - aE)^2 + Q) - 2 r Delta, P = E (r^2 + a^2) - a L_z */
    double Delta = rp * rp - 2.0 * M * rp + a * a;
    double P = E * (rp * rp + a * a) - a * Lz;
    F[1] = 2.0 * P * 2.0 * E * rp - (2.0 * rp - 2.0 * M) * (rp * rp + (Lz - a * E) * (Lz - a * E) + Q) -
           2.0 * rp * Delta;
  } else {
    F[1] = orc_radial_potential(M, a, E, Lz, Q, ra);
  }
}

int orc_bound_orbit_solve(double M, double a, double rp, double e, double iota, double* E_out,
                          double* Lz_out, double* Q_out, double* r3_out) {
  int circ = e < 1e-6;
  double ra = circ ? rp : rp * (1.0 + e) / (1.0 - e);
  double ci = cos(iota), si = sin(iota);
  double pM = rp * (1.0 + e) / M;
  double den = pM - 3.0 - e * e;
  double E, L;
  if (den > 0.05) {
    E = sqrt((pM - 2.0 - 2.0 * e) * (pM - 2.0 + 2.0 * e) / (pM * den));
    L = M * pM / sqrt(den);
  } else {
    E = 0.95;
    L = 4.0 * M;
  }
  int ok = 0;
  for (int it = 0; it < 200; ++it) {
    double F[2], Fe[2], Fl[2];
    bound_residual(M, a, rp, ra, circ, ci, si, E, L, F);
    double scale = rp * rp * rp * rp;
    if (fabs(F[0]) < 1e-14 * scale && fabs(F[1]) < 1e-14 * scale) { ok = 1; break; }
    double dE = 1e-7 * fmax(fabs(E), 1e-3), dL = 1e-7 * fmax(fabs(L), 1e-3);
    bound_residual(M, a, rp, ra, circ, ci, si, E + dE, L, Fe);
    bound_residual(M, a, rp, ra, circ, ci, si, E, L + dL, Fl);
    double J00 = (Fe[0] - F[0]) / dE, J10 = (Fe[1] - F[1]) / dE;
    double J01 = (Fl[0] - F[0]) / dL, J11 = (Fl[1] - F[1]) / dL;
    double det = J00 * J11 - J01 * J10;
    if (det == 0.0 || !isfinite(det)) break;
    double sE = -(J11 * F[0] - J01 * F[1]) / det;
    double sL = -(-J10 * F[0] + J00 * F[1]) / det;
    /* damping: keep the update within 10% of the current values */
    double lim = 0.1;
    double fac = 1.0;
    if (fabs(sE) > lim * fabs(E)) fac = fmin(fac, lim * fabs(E) / fabs(sE));
    if (fabs(sL) > lim * fabs(L)) fac = fmin(fac, lim * fabs(L) / fabs(sL));
    E += fac * sE;
    L += fac * sL;
  }
  if (!ok) {
    /* one last residual check: Newton may stop at the tolerance edge */
    double F[2];
    bound_residual(M, a, rp, ra, circ, ci, si, E, L, F);
    double scale = rp * rp * rp * rp;
    if (!(fabs(F[0]) < 1e-11 * scale && fabs(F[1]) < 1e-11 * scale)) return 1;
  }
  if (!(E > 0.0 && E < 1.0) || !(L > 0.0)) return 2;
  double Lz = L * ci, Q = L * L * si * si;
  /* remaining roots of R(r) = (E^2 - 1)(r - ra)(r - rp)(r - r3)(r - r4):
   * sum of roots 2M/(1 - E^2), product a^2 Q/(1 - E^2) */
  double S = 2.0 * M / (1.0 - E * E) - ra - rp;
  double P = a * a * Q / ((1.0 - E * E) * ra * rp);
  double disc = S * S - 4.0 * P;
  double r3 = disc >= 0.0 ? 0.5 * (S + sqrt(disc)) : -INFINITY;
  if (r3_out) *r3_out = r3;
  if (r3 >= rp) return 3;
  if (!circ && !(orc_radial_potential(M, a, E, Lz, Q, 0.5 * (rp + ra)) > 0.0)) return 4;
  *E_out = E;
  *Lz_out = Lz;
  *Q_out = Q;
  return 0;
}

/* Seeded generic bound-orbit sampler.  Particle `index` draws its spin
 * a = a_max U(counter index*256) (or takes a = a_max when spin_fixed), then candidates j = 0..63 with
 *   rp = r_lo + (10M - r_lo) U(index*256 + 4j + 1),  r_lo = ISCO_prograde(a) + 0.5M,
 *   e = 0.7 U(index*256 + 4j + 2),  iota = pi U(index*256 + 4j + 3),
 * and keeps the first bound, stable one.  State: x = (0, rp, pi/2, 0),
 * p = (-E, 0, +sqrt(Q), L_z), u = g^{-1} p.  Returns the accepted candidate
 * index, or -1 when all 64 were rejected (then the prograde circular
 * equatorial orbit at r = 10M is used).  cand = (rp, e, iota, attempts). */
int orc_bound_sample(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t index,
                     double* a_out, double y[8], double cand[4]) {
  uint64_t base = index * 256u;
  double a = spin_fixed ? a_max : a_max * orc_uniform(seed, base);
  double r_lo = orc_isco_bardeen(M, a, 1) + 0.5 * M, r_hi = 10.0 * M;
  *a_out = a;
  for (int j = 0; j < 64; ++j) {
    double rp = r_lo + (r_hi - r_lo) * orc_uniform(seed, base + 4u * j + 1u);
    double e = 0.7 * orc_uniform(seed, base + 4u * j + 2u);
    double iota = M_PI * orc_uniform(seed, base + 4u * j + 3u);
    double E, Lz, Q, r3;
    if (orc_bound_orbit_solve(M, a, rp, e, iota, &E, &Lz, &Q, &r3) == 0) {
      double x[4] = {0.0, rp, M_PI / 2.0, 0.0};
      double p[4] = {-E, 0.0, sqrt(Q), Lz};
      momenta_to_state(M, a, x, p, y);
      if (cand) { cand[0] = rp; cand[1] = e; cand[2] = iota; cand[3] = j + 1; }
      return j;
    }
  }
  orc_circular_state(M, a, r_hi, 1, y);
  if (cand) { cand[0] = r_hi; cand[1] = 0.0; cand[2] = 0.0; cand[3] = 64; }
  return -1;
}

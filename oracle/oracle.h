/*
 * oracle.h -- plain, slow FP64 CPU oracle for geodesics of the Kerr and
 * Schwarzschild black holes in Boyer-Lindquist coordinates, integrated with
 * classical fixed-step RK4 (Quiroga, "MALBEC: a new CUDA-C ray-tracer in
 * General Relativity", arXiv:1803.08320).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: every quantity here is
 * written out from its definition, in scalar double precision, in the order
 * the paper (or the textbook result it names) states it.
 *
 * Conventions (all functions):
 *   - geometrised units G = c = 1; mass M > 0, spin a with |a| <= M;
 *   - coordinates x^mu = (t, r, theta, phi), indices 0..3 in that order;
 *   - a state y[8] = (x^0..x^3, u^0..u^3) with u^mu = dx^mu/dlambda;
 *   - 4x4 tensors are row-major double[16]; a derivative array dg[64] holds
 *     dg[s*16 + m*4 + n] = d g_{mn} / d x^s;
 *   - covariant p_t = -E (the paper prints +E in its p_t columns; the helper
 *     orc_paper_to_state flips that sign).
 */
#ifndef MALBEC_ORACLE_H
#define MALBEC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* fate codes (an interface both sides must agree on; values fixed by the ABI) */
#define ORC_FATE_CAPTURED 1
#define ORC_FATE_ESCAPED 2
#define ORC_FATE_CAPPED 3
#define ORC_FATE_NONFINITE 4
/* validity flag or-ed into the fate of an ESCAPED or CAPPED ray: the norm
 * g(u,u) at the end departs from its value at the start by more than
 * ORC_NORM_DRIFT_TOL max(E^2, |g(u,u)|) (E and g(u,u) of the start state); the
 * flow keeps g(u,u) constant (Sec. 2, eq. geo), so such an end state is not a
 * solution to trust.  A CAPTURED ray ends at the capture radius, where the BL
 * norm is dominated by u^t ~ 1/Delta, and is never flagged. */
#define ORC_FATE_DRIFTED 0x80
#define ORC_NORM_DRIFT_TOL 1e-3

typedef struct {
  double eps_hor;      /* captured when r <= (1+eps_hor) r_+ */
  double r_esc;        /* escaped when r >= r_esc */
  uint32_t n_steps_cap;/* capped after this many steps */
  double dl;           /* fixed step, used when dl_r_scale == 0 */
  double dl_r_scale;   /* if > 0: h_n = dl_r_scale * r_n (r at the step start) */
  uint32_t form;       /* 0: the geodesic equation in (x, u) (Sec. 2, eq. geo);
                          1: the canonical equations in (x, p) (Sec. 2, eq. Ham)
                             with g of eq. kerr;
                          2: the same equations with g built from the lapse,
                             shift and 3-metric of eq. ADM */
  uint32_t method;     /* 0: classical RK4 with the fixed step rule above;
                          1: Dormand-Prince 5(4) with step-size control:
                             first trial step dl (or dl_r_scale r0 if dl = 0),
                             every step at most dl_r_scale r when dl_r_scale > 0,
                             local error norm against atol + rtol |y|, step
                             factor 0.9 err^(-1/5) taken down to the grid 2^(j/4);
                             n_steps_cap and the step count then count attempts */
  double rtol, atol;   /* tolerances of method 1 (atol > 0) */
  double rhs_noise;    /* test-only (0 = off): every right-hand-side component is
                          multiplied by 1 +- rhs_noise, the sign drawn from
                          SplitMix64 (seeded with the bits of rhs_noise) on a
                          per-ray counter of evaluations -- a
                          rounding-sized perturbation that measures how much a
                          ray's result depends on the rounding of its steps */
} orc_term;

/* -------- geometry (Sec. 2, eq. kerr) -------- */
double orc_r_plus(double M, double a);
void orc_metric(double M, double a, double r, double th, double g[16]);
void orc_metric_derivs(double M, double a, double r, double th, double dg[64]);
void orc_inverse_metric(double M, double a, double r, double th, double gi[16]);
void orc_christoffel(double M, double a, double r, double th, double G[64]);
void orc_adm(double M, double a, double r, double th, double* alpha, double* beta_phi, double gamma[3]);
/* d/dr (k = 0) and d/dtheta (k = 1) of alpha, beta^phi and gamma_ii
 * (dgamma[i * 2 + k], i = rr, thth, phph) */
void orc_adm_derivs(double M, double a, double r, double th, double dalpha[2], double dbeta_phi[2],
                    double dgamma[6]);
/* g_{mn} and d_s g_{mn} assembled from the ADM quantities (eq. ADM) */
void orc_adm_metric(double M, double a, double r, double th, double g[16]);
void orc_adm_metric_derivs(double M, double a, double r, double th, double dg[64]);
void orc_invert4(const double A[16], double Ai[16]);  /* Gauss-Jordan, partial pivoting */

/* -------- equations of motion -------- */
void orc_rhs(double M, double a, const double y[8], double f[8]);          /* geodesic eq., Christoffel form */
void orc_rhs_hamiltonian(double M, double a, const double z[8], double f[8]); /* eq. Ham, state (x^mu, p_mu) */
void orc_rhs_adm(double M, double a, const double z[8], double f[8]);         /* eq. Ham with g from eq. ADM */
double orc_hamiltonian_adm(double M, double a, const double z[8]);          /* H = g^{mn} p_m p_n / 2 */
void orc_rk4_linear_test(double lam, double h, int nsteps, double* y);   /* RK4 on y' = lam*y */
void orc_rk4_step(double M, double a, double h, double y[8]);
void orc_rk4_step_hamiltonian(double M, double a, double h, double z[8]);
void orc_rk4_step_adm(double M, double a, double h, double z[8]);
/* Dormand-Prince 5(4) tableau: c[7], a[7*7] row-major (strictly lower), the
 * fifth-order weights b[7] and the embedded fourth-order weights bhat[7]. */
void orc_dopri5_tableau(double c[7], double a[49], double b[7], double bhat[7]);
/* One Dormand-Prince attempt of size h on y' = lam y (y scalar): y5, and the
 * error estimate y5 - y4 in *err. */
void orc_dopri5_linear_test(double lam, double h, double y0, double* y5, double* err);

/* -------- integration with termination (Sec. 5) -------- */
int orc_trace_one(double M, double a, const double y0[8], const orc_term* t,
                  double y[8], double* lambda, uint32_t* steps,
                  double* traj, uint32_t stride);
/* n rays, SoA in/out (component c of ray i at [c*n + i]); a_per_ray may be NULL.
 * Outputs: y_out 8*n, lambda n, inv0 4*n (start), inv1 4*n (end), steps n, fate n.
 * traj (optional, NULL to skip): n * (cap/stride + 1) * 8 doubles, ray-major.
 * nthreads <= 0: use the OpenMP default.  Returns the thread count used. */
int orc_trace_many(double M, double a, const double* a_per_ray, const double* ics, uint64_t n,
                   const orc_term* t, double* y_out, double* lambda, double* inv0, double* inv1,
                   uint32_t* steps, uint8_t* fate, double* traj, uint32_t stride, int nthreads);

/* -------- conserved quantities -------- */
void orc_invariants(double M, double a, const double y[8], double inv[4]); /* E, L_z, Q, norm */

/* -------- initial conditions -------- */
void orc_paper_to_state(double M, double a, const double xp[8], double y[8]);
void orc_state_to_momenta(double M, double a, const double y[8], double p[4]);
void orc_bl_to_cartesian(double a, double r, double th, double ph, double xyz[3]);
void orc_schw_circular(double M, double r, double* E, double* L);          /* eqs. COrbit, COrbit2 */
void orc_schw_gralorbits(double k, double M, double* pt, double* pphi);     /* eq. gralorbits */
void orc_kerr_circular_paper(double M, double a, double r, int sgn, double* E, double* L); /* eqs. energia, momento as printed */
void orc_kerr_circular_bardeen(double M, double a, double r, int prograde, double* E, double* L);
double orc_kerr_omega(double M, double a, double r, double pt_paper, double pphi); /* eq. omega */
double orc_isco_bardeen(double M, double a, int prograde);
double orc_isco_paper_literal(double M, double a, int sgn);                /* eq. iscokerr as printed */
double orc_dEdr_numeric_root(double M, double a, int prograde, double r_lo, double r_hi);
double orc_photon_orbit(double M, double a, int prograde);
void orc_circular_state(double M, double a, double r, int prograde, double y[8]);
void orc_camera_ic(double M, double a, double r_o, double th_o, double fov_half,
                   uint32_t nx, uint32_t ny, uint64_t pix, double y[8]);
double orc_critical_curve_distance(double M, double a, double th_o, double alpha, double beta);
void orc_critical_curve_polyline(double M, double a, double th_o, int n, double* alpha, double* beta);

/* -------- generic bound orbits (counter-based sampler) -------- */
uint64_t orc_splitmix64(uint64_t seed, uint64_t counter);
double orc_uniform(uint64_t seed, uint64_t counter);
int orc_bound_orbit_solve(double M, double a, double rp, double e, double iota,
                          double* E, double* Lz, double* Q, double* r3);
int orc_bound_sample(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t index,
                     double* a_out, double y[8], double cand[4]);
double orc_radial_potential(double M, double a, double E, double Lz, double Q, double r);

#ifdef __cplusplus
}
#endif
#endif

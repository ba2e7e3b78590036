// camera.cuh -- backward null-ray camera: pixel -> initial state.
// Not in the paper (its initial conditions come from a file, Sec. 5); impact
// parameters after Bardeen (1973).  Pixel p = j*nx + i has
//   alpha = -fov + 2 fov (i + 1/2)/nx,  beta = -fov + 2 fov (j + 1/2)/ny;
// the photon arriving at the observer has E = 1, L_z = -alpha sin(incl),
// Q = beta^2 + cos^2(incl) (alpha^2 - a^2), p_th = sign(beta) sqrt(Theta(incl)),
// Theta = Q + a^2 cos^2 - L_z^2 cot^2, p_r = +sqrt(R(r_obs))/Delta(r_obs),
// R = ((r^2 + a^2) E - a L_z)^2 - Delta (Q + (L_z - a E)^2).  It is traced
// backward by integrating forward in lambda with the momentum reversed:
// u = g^{-1}(E, -p_r, -p_th, -L_z), g^{-1} at the observer precomputed.
#pragma once
#include "internal.h"

namespace malbec {

// Claim order of a whole-image trace: the k-th ray taken from the work queue
// is the pixel of column rank k / ny (columns by increasing |alpha|, the
// centre first) and row k % ny.  |L_z| = |alpha| sin(incl) is smallest in the
// centre columns; those rays pass closest to the polar axis and take the
// most steps (up to 30x the mean), so starting them first keeps them from
// setting the end of the launch.  A permutation of the pixels: every pixel's
// result is unchanged.
__device__ __forceinline__ uint64_t camera_claim_pixel(const CameraConst& c, uint64_t k) {
  const uint64_t rank = k / c.ny, row = k - rank * c.ny;
  const uint64_t mid = c.nx / 2;
  uint64_t col;
  if (c.nx & 1u)  // odd: mid, mid - 1, mid + 1, mid - 2, ...
    col = rank == 0 ? mid : ((rank & 1u) ? mid - (rank + 1) / 2 : mid + rank / 2);
  else            // even: mid - 1, mid, mid - 2, mid + 1, ...
    col = (rank & 1u) ? mid + rank / 2 : mid - 1 - rank / 2;
  return row * c.nx + col;
}

__device__ __forceinline__ void camera_state(const CameraConst& c, double a, uint64_t pix, double y[8]) {
  const uint64_t i = pix % c.nx, j = pix / c.nx;
  const double alpha = -c.fov_half + 2.0 * c.fov_half * ((double)i + 0.5) / (double)c.nx;
  const double beta = -c.fov_half + 2.0 * c.fov_half * ((double)j + 0.5) / (double)c.ny;
  const double L = -alpha * c.so;
  const double co2 = c.co * c.co;
  const double Q = beta * beta + co2 * (alpha * alpha - a * a);
  const double Theta = Q + a * a * co2 - L * L * co2 / (c.so * c.so);
  const double pth = (beta >= 0.0 ? 1.0 : -1.0) * sqrt(fmax(Theta, 0.0));
  const double P = c.r2a2_o - a * L;
  const double R = P * P - c.Delta_o * (Q + (L - a) * (L - a));
  const double pr = sqrt(fmax(R, 0.0)) / c.Delta_o;
  y[0] = 0.0;
  y[1] = c.r_obs;
  y[2] = c.incl;
  y[3] = 0.0;
  y[4] = c.gtt - c.gtp * L;
  y[5] = -c.grr * pr;
  y[6] = -c.ghh * pth;
  y[7] = c.gtp - c.gpp * L;
}

}  // namespace malbec

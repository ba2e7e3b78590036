// ic.cu -- initial-data and invariant kernels (FP64).
//
//  - circular equatorial orbits: Schwarzschild E, L of Sec. 4 (eqs. COrbit,
//    COrbit2) for a = 0, Bardeen-Press-Teukolsky closed forms for Kerr (the
//    paper's eqs. energia/momento with the co-/counter-rotating labels as in
//    its tables);
//  - backward camera pixels (Bardeen 1973 impact parameters);
//  - generic bound Kerr orbits drawn with the SplitMix64 counter-based
//    generator and solved by Newton's method with the analytic Jacobian of
//    the radial potential R(r);
//  - the paper's own initial-condition rows (p_t column = E) to states;
//  - E, L_z, Q, g(u,u) of arrays of states.
#include <math.h>

#include "bound.cuh"
#include "camera.cuh"
#include "geodesic.cuh"
#include "internal.h"

namespace malbec {
namespace {

constexpr int kTPB = 128;

__global__ void ic_circular_kernel(double M, double a, const double* __restrict__ radii, uint64_t n,
                                   int prograde, double* __restrict__ ics) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double r = radii[i];
  const double sg = prograde ? 1.0 : -1.0;
  double E, L;
  if (a == 0.0) {
    // Sec. 4 eqs. COrbit, COrbit2
    E = sqrt((r - 2.0 * M) * (r - 2.0 * M) / (r * (r - 3.0 * M)));
    L = sg * sqrt(M * r * r / (r - 3.0 * M));
  } else {
    circular_EL(M, a, r, sg, &E, &L);
  }
  const double p[4] = {-E, 0.0, 0.0, L};
  double u[4];
  raise_momenta(M, a, r, kHalfPi, p, u);
  const double y[8] = {0.0, r, kHalfPi, 0.0, u[0], u[1], u[2], u[3]};
#pragma unroll
  for (int c = 0; c < 8; ++c) ics[(size_t)c * n + i] = y[c];
}

__global__ void ic_camera_kernel(double M, double a, CameraConst cam, const uint64_t* __restrict__ pixels,
                                 uint64_t n, double* __restrict__ ics) {
  const uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double y[8];
  camera_state(cam, a, pixels[k], y);
  (void)M;
#pragma unroll
  for (int c = 0; c < 8; ++c) ics[(size_t)c * n + k] = y[c];
}


__global__ void ic_bound_kernel(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t index0, uint64_t n,
                                double* __restrict__ ics, double* __restrict__ spins, int32_t* __restrict__ accepted) {
  const uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  double y[8], a;
  const int acc = bound_sample(M, a_max, spin_fixed, seed, index0 + k, y, &a);
#pragma unroll
  for (int c = 0; c < 8; ++c) ics[(size_t)c * n + k] = y[c];
  spins[k] = a;
  accepted[k] = acc;
}

__global__ void invariants_kernel(double M, double a, const double* __restrict__ a_per_ray,
                                  const double* __restrict__ states, uint64_t n, double* __restrict__ inv) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double y[8], v[4];
#pragma unroll
  for (int c = 0; c < 8; ++c) y[c] = states[(size_t)c * n + i];
  invariants64(M, a_per_ray ? a_per_ray[i] : a, y, v);
#pragma unroll
  for (int c = 0; c < 4; ++c) inv[(size_t)c * n + i] = v[c];
}

// The paper's initial-condition rows (Sec. 5: t, r, theta, phi and the
// momenta p_t, p_r, p_theta, p_phi, with the p_t column holding E > 0) to
// states (x, u): p = (-E, p_r, p_theta, p_phi), u = g^{-1} p (eq. kerr).
__global__ void ic_from_paper_kernel(double M, double a, const double* __restrict__ a_per_ray,
                                     const double* __restrict__ rows, uint64_t n, double* __restrict__ ics) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double z[8], u[4];
#pragma unroll
  for (int c = 0; c < 8; ++c) z[c] = rows[(size_t)c * n + i];
  z[4] = -z[4];
  raise_momentum(M, a_per_ray ? a_per_ray[i] : a, z, u);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    ics[(size_t)c * n + i] = z[c];
    ics[(size_t)(4 + c) * n + i] = u[c];
  }
}

unsigned grid_for(uint64_t n) { return (unsigned)((n + kTPB - 1) / kTPB); }

}  // namespace

cudaError_t launch_ic_circular(double M, double a, const double* radii, uint64_t n, int prograde, double* ics,
                               cudaStream_t stream) {
  ic_circular_kernel<<<grid_for(n), kTPB, 0, stream>>>(M, a, radii, n, prograde, ics);
  return cudaGetLastError();
}

cudaError_t launch_ic_camera(double M, double a, const CameraConst& cam, const uint64_t* pixels, uint64_t n,
                             double* ics, cudaStream_t stream) {
  ic_camera_kernel<<<grid_for(n), kTPB, 0, stream>>>(M, a, cam, pixels, n, ics);
  return cudaGetLastError();
}

cudaError_t launch_ic_bound(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t index0, uint64_t n,
                            double* ics, double* spins, int32_t* accepted, cudaStream_t stream) {
  ic_bound_kernel<<<grid_for(n), kTPB, 0, stream>>>(M, a_max, spin_fixed, seed, index0, n, ics, spins, accepted);
  return cudaGetLastError();
}

cudaError_t launch_ic_from_paper(double M, double a, const double* a_per_ray, const double* rows, uint64_t n,
                                 double* ics, cudaStream_t stream) {
  ic_from_paper_kernel<<<grid_for(n), kTPB, 0, stream>>>(M, a, a_per_ray, rows, n, ics);
  return cudaGetLastError();
}

cudaError_t launch_invariants(double M, double a, const double* a_per_ray, const double* states, uint64_t n,
                              double* inv, cudaStream_t stream) {
  invariants_kernel<<<grid_for(n), kTPB, 0, stream>>>(M, a, a_per_ray, states, n, inv);
  return cudaGetLastError();
}

}  // namespace malbec

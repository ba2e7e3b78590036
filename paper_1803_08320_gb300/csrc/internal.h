// internal.h -- host-side declarations shared by the translation units of
// libmalbec.so (not part of the public ABI; see include/malbec.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/malbec.h"

namespace malbec {

enum Source : int { kSrcStates = 0, kSrcCamera = 1, kSrcJobs = 2, kSrcServe = 3 };
enum Sink : int { kSinkFinal = 0, kSinkStrided = 1, kSinkCamera = 2, kSinkJobs = 3 };

// Per-image constants of the backward camera (computed on the host in FP64).
struct CameraConst {
  double r_obs, incl, fov_half;
  uint32_t nx, ny;
  double so, co;             // sin, cos of the inclination
  double Delta_o, r2a2_o;    // Delta(r_obs), r_obs^2 + a^2
  double gtt, gtp, gpp, grr, ghh;  // inverse metric at the observer
};

// One job (bundle) of the multi-job trace kernel, resident in device memory.
struct JobDesc {
  int32_t kind;  // MALBEC_BUNDLE_*
  uint32_t cap;
  uint64_t n;
  uint64_t job_id;  // serving: the id whose slot this is (0 = empty)
  double M, a, eps_hor, r_esc, dl, dl_r_scale;
  uint64_t seed;
  uint32_t form, method;  // MALBEC_FORM_*, MALBEC_METHOD_* (every job of a launch has the same)
  double rtol, atol;      // MALBEC_METHOD_DOPRI5 tolerances of this job
  CameraConst cam;
  const double* ics;
  // outputs: FINAL layout (states, bound) or camera layout (camera)
  double* y_out;
  double* lambda_out;
  double* inv0_out;
  double* inv1_out;
  uint32_t* steps_out;
  uint8_t* fate_out;
  double* theta_out;
  double* phi_out;
};

struct JobCounter {
  unsigned long long next;  // rays handed out
  unsigned long long done;  // rays finished
};

struct TraceParams {
  // black hole
  double M, a;
  const double* a_per_ray;
  // step rule / termination
  double eps_hor, r_esc, dl, dl_r_scale;
  uint32_t cap;
  // rays
  const double* ics;  // SoA [8][n] (kSrcStates)
  uint64_t n;
  CameraConst cam;    // kSrcCamera
  // outputs (kSinkFinal / kSinkStrided)
  double* y_out;
  double* lambda_out;
  double* inv0_out;
  double* inv1_out;
  uint32_t* steps_out;
  uint8_t* fate_out;
  void* traj;
  uint32_t stride;
  uint64_t n_samples;
  int traj_cartesian;  // samples are (t, x, y, z) of eq. coord instead of the state
  // outputs (kSinkCamera)
  double* theta_out;
  double* phi_out;
  // FP32_MIXED FP64 zone (malbec_mixed_zone) and the batching of zone steps
  double zone_horizon, zone_photon, zone_pole;
  int zone_batch, zone_wait;
  int exchange;       // FP32_MIXED: block ray exchange on (1) / off (0)
  uint64_t zone_wait_ns;  // the zone warp's longest wait for its block (device clock)
  uint32_t form;      // MALBEC_FORM_*
  uint32_t method;    // MALBEC_METHOD_*
  double rtol, atol;  // MALBEC_METHOD_DOPRI5 tolerances
  // work queue (scratch, zeroed before launch)
  unsigned long long* head;
  // multi-job source: job table, per-job counters (zeroed), longest-first
  // job order and the cursor into it (zeroed)
  const JobDesc* jobs;
  JobCounter* job_ctr;
  const uint32_t* job_order;
  uint32_t n_jobs;
  unsigned int* job_cursor;
  // serving source: `jobs`/`job_ctr` form a ring of n_jobs slots (slot =
  // job_id % n_jobs); the active list, the stop flag and the completion
  // flags live in mapped host memory
  const volatile uint64_t* active_ids;
  const volatile uint32_t* active_count;
  const volatile uint32_t* stop_flag;
  volatile uint64_t* done_flags;
  uint32_t max_active;
  uint64_t idle_ns;
  // request loop: warps that have been idle for idle_ns park here (low 32
  // bits count them); the kernel leaves only when every warp is parked (the
  // warp that sees it sets bit 63, closing), never part of it
  unsigned long long* park;
  // launch shape
  int refill_min;  // refill when at least this many lanes of a warp are idle
  // always 0 (every TraceParams is zeroed): ANDed with threadIdx.x it gives
  // FP64 kernels a zero the compiler cannot fold or prove warp-uniform, which
  // keeps their constant operands in per-thread registers (make_bh)
  unsigned long long lane_zero;
};

struct LaunchShape {
  int threads_per_block;
  int blocks;
};

// trace.cu
cudaError_t launch_trace(const TraceParams& p, bool kerr, bool mixed, Source src, Sink sink,
                         const LaunchShape& shape, cudaStream_t stream);
// trace_dopri.cu: the Dormand-Prince kernel for (mixed, src, sink, form), or
// nullptr if there is none
const void* pick_dopri(bool mixed, Source src, Sink sink, int form);
// resident blocks per SM of the geodesic RK4 kernel of (kerr, mixed, src,
// sink), with (banks) or without the FP32_MIXED block ray exchange
int trace_max_blocks_per_sm(bool kerr, bool mixed, Source src, Sink sink, bool banks, int threads_per_block,
                            int form = MALBEC_FORM_GEODESIC, int method = MALBEC_METHOD_RK4);
// total of the device-wide counter of zone-warp waits that ran out (current device)
cudaError_t read_wait_timeouts(unsigned long long* total);

// ic.cu
cudaError_t launch_ic_circular(double M, double a, const double* radii, uint64_t n, int prograde,
                               double* ics, cudaStream_t stream);
cudaError_t launch_ic_camera(double M, double a, const CameraConst& cam, const uint64_t* pixels,
                             uint64_t n, double* ics, cudaStream_t stream);
cudaError_t launch_ic_bound(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t index0,
                            uint64_t n, double* ics, double* spins, int32_t* accepted,
                            cudaStream_t stream);
cudaError_t launch_ic_from_paper(double M, double a, const double* a_per_ray, const double* rows, uint64_t n,
                                 double* ics, cudaStream_t stream);
cudaError_t launch_invariants(double M, double a, const double* a_per_ray, const double* states,
                              uint64_t n, double* inv, cudaStream_t stream);

// api.cu
int set_cuda_error(cudaError_t e);
void fill_zone(TraceParams& p);
int check_metric(const malbec_metric& m);
int check_term(const malbec_term& t, const malbec_metric& m);
int check_method_precision(const malbec_term& t, malbec_precision prec, bool mixed_ok = false);
int choose_shape(bool kerr, bool mixed, Source src, Sink sink, uint64_t n, LaunchShape* shape, int* refill_min,
                 int form = MALBEC_FORM_GEODESIC, int method = MALBEC_METHOD_RK4);
int choose_shape_cfg(bool kerr, bool mixed, Source src, Sink sink, uint64_t n, const malbec_launch_config& cfg,
                     LaunchShape* shape, int* refill_min, int form = MALBEC_FORM_GEODESIC,
                     int method = MALBEC_METHOD_RK4);
int check_camera_desc(const malbec_metric& m, const malbec_camera* cam, const malbec_term* t);

// bundles.cu
int validate_job(const malbec_bundle& b, malbec_precision prec);
void fill_job_desc(const malbec_bundle& b, malbec_precision prec, void* out, uint64_t job_id, JobDesc* J,
                   double* cost);
CameraConst make_camera_const(double M, double a, const malbec_camera& cam);

}  // namespace malbec

/*
 * malbec.h -- C ABI of libmalbec.so, a single-GPU (GB300, sm_103a) library
 * that integrates timelike and null geodesics of the Schwarzschild and Kerr
 * black holes in Boyer-Lindquist (BL) coordinates with classical fixed-step
 * RK4, one ray per GPU thread (Quiroga, "MALBEC: a new CUDA-C ray-tracer in
 * General Relativity", arXiv:1803.08320).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Units G = c = 1.  Coordinates x^mu = (t, r, theta, phi), index order
 *    0..3.  A state is y = (x^0..x^3, u^0..u^3), u^mu = dx^mu/dlambda.
 *  - Arrays of states are structure-of-arrays: component c of ray i lives at
 *    ptr[c * n + i] (c = 0..7).
 *  - Pointers documented as "device" must point to memory of the current CUDA
 *    device (e.g. tensors allocated by PyTorch).  The caller owns all such
 *    memory; the library never frees it.  Pointers documented as "host" are
 *    ordinary host memory.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and the call returns without waiting, unless stated otherwise.
 *  - Return value: MALBEC_OK (0) or a negative MALBEC_E* code.  Invalid
 *    arguments are rejected before any work is enqueued.  Per-ray outcomes
 *    (capture, escape, cap, non-finite) are fate codes in the output, not
 *    call errors.  A CUDA launch or allocation failure returns MALBEC_ECUDA;
 *    malbec_last_cuda_error() gives the CUDA error string.
 *  - Every entry point is thread-safe with respect to other entry points; two
 *    calls on different streams run concurrently on the GPU.
 */
#ifndef MALBEC_H
#define MALBEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* malbec_stream; /* == cudaStream_t */

/* ---------------------------------------------------------------- errors */
#define MALBEC_OK 0
#define MALBEC_EINVAL (-1)    /* bad argument (a >= M, M <= 0, a camera observer inside the capture
                                 radius, a NaN parameter, n == 0, ...); device initial states are
                                 not read on the host: a bad ray ends with its own fate */
#define MALBEC_ENOMEM (-2)    /* over the HBM budget, or a device allocation failed */
#define MALBEC_EBUSY (-3)     /* admission queue full: retry later */
#define MALBEC_ETIMEDOUT (-4) /* a bounded device-side wait gave up */
#define MALBEC_ECUDA (-5)     /* CUDA runtime error; see malbec_last_cuda_error() */
#define MALBEC_ENOTFOUND (-6) /* unknown job id */
#define MALBEC_ESCRATCH (-7)  /* a no-allocation call needs more scratch than its static block holds */

/* Human-readable text of a MALBEC_* code (static storage, never NULL). */
const char* malbec_strerror(int code);
/* Text of the last CUDA error seen by this thread (static storage). */
const char* malbec_last_cuda_error(void);

/* ---------------------------------------------------------------- fates */
/* Per-ray termination, tested after every completed RK4 step in this order
 * (Sec. 5 of the paper stops a thread at the horizon, r <= 1 + sqrt(1 - a^2)
 * for M = 1; this library generalises it to (1 + eps_hor) r_+ and adds the
 * escape radius, a non-finite check and the step cap):
 *   CAPTURED  r <= (1+eps_hor) r_+ at the new state or at one of the step's
 *             intermediate RK4 stage points (r_+ = M + sqrt(M^2 - a^2));
 *   NONFINITE some component of the new state is NaN or infinite;
 *   ESCAPED   r >= r_esc;
 *   CAPPED    n_steps_cap steps taken. */
#define MALBEC_FATE_CAPTURED 1
#define MALBEC_FATE_ESCAPED 2
#define MALBEC_FATE_CAPPED 3
#define MALBEC_FATE_NONFINITE 4
/* Validity flag, or-ed into the fate byte of every output (state arrays,
 * cameras, bundles, server jobs): the ray's norm g(u,u), evaluated in FP64 at
 * its end, departs from its value at the start by more than
 *   MALBEC_NORM_DRIFT_TOL * max(E^2, |g(u,u)|)   (E = -p_t, both at the start).
 * The geodesic flow keeps g(u,u) exactly constant (Sec. 2 eq. geo: 0 for
 * null rays, -1 for timelike ones), so such a ray's end state and angles are
 * not a solution to trust: typically a fixed step much too long for a
 * passage next to the polar axis, where the BL right-hand side diverges (the
 * fixed-step RK4 of the Kerr a = 0.9 camera at 80 degrees flags about 4.5% of
 * its escaped rays; about a third of those have blown up, |dg| > E^2).
 * Set on ESCAPED and CAPPED rays only, the ones whose end state and angles
 * are results: a CAPTURED ray ends at the capture radius, where u^t ~ 1/Delta
 * grows without bound in BL coordinates and its norm says nothing about the
 * path, and a NONFINITE ray is already invalid.
 * fate & MALBEC_FATE_MASK is the termination itself. */
#define MALBEC_FATE_DRIFTED 0x80
#define MALBEC_FATE_MASK 0x7f
#define MALBEC_NORM_DRIFT_TOL 1e-3

/* ---------------------------------------------------------------- parameters */
/* Black hole.  Kerr metric in BL coordinates, Sec. 2 eq. kerr; a = 0 is
 * Schwarzschild (Sec. 4) and selects the specialised Schwarzschild kernel.
 * Requires M > 0 and 0 <= a < M (Sec. 2 restricts to a <= M; a = M is
 * rejected because r_+ = M makes the capture radius degenerate).
 * a_per_ray: optional device array of n spins (overrides a per ray; each
 * must satisfy 0 <= a_i < M; not validated on the host -- a ray with an
 * invalid spin ends NONFINITE). */
typedef struct {
  double M;
  double a;
  const double* a_per_ray;
} malbec_metric;

/* Step rule and termination.  The step is h = dl, or h = dl_r_scale * r_n
 * (r at the start of the step, held for all four stages) when
 * dl_r_scale > 0.  The paper uses a fixed h (Sec. 6).  Requires eps_hor >= 0,
 * r_esc > (1+eps_hor) r_+, and a finite positive step (for DOPRI5 below,
 * dl >= 0 when dl_r_scale > 0).
 * form: the equations RK4 integrates --
 *   MALBEC_FORM_GEODESIC     (0) the geodesic equation in (x^mu, u^mu),
 *                            du/dl = -Gamma u u (Sec. 2, eq. geo);
 *   MALBEC_FORM_HAMILTONIAN  (1) the canonical equations in (x^mu, p_mu),
 *                            p = g u, H = g^{ab} p_a p_b / 2 (Sec. 2, eq. Ham):
 *                            the paper's own form; p_t and p_ph (-E and L_z)
 *                            stay exactly constant.  FP64 and FP32_MIXED
 *                            (same FP64 zones); every entry point (bundles:
 *                            one persistent launch per (form, method) class;
 *                            servers: one class per server).
 *   MALBEC_FORM_ADM          (2) the same canonical equations with H written
 *                            through the lapse alpha, shift beta^ph and
 *                            spatial metric gamma_ij of the 3+1 line element
 *                            (Sec. 2, eq. ADM; Kerr's alpha, beta, gamma as
 *                            the paper gives them after eq. coord) and their
 *                            r- and theta-derivatives.  The right-hand side
 *                            holds for any stationary, axisymmetric, circular
 *                            metric; Kerr is the metric supplied.  Same entry
 *                            points and precisions as form 1; the same flow,
 *                            so its RK4 map equals form 1's up to rounding.
 * Inputs and outputs are (x, u) states in every form; the geodesic and the
 * canonical maps agree to O(h^4) per unit lambda.
 * method: the integrator --
 *   MALBEC_METHOD_RK4     (0) classical fourth-order Runge-Kutta with the
 *                         step rule above (the paper's, Sec. 5);
 *   MALBEC_METHOD_DOPRI5  (1) the Dormand-Prince 5(4) embedded pair
 *                         (Dormand & Prince 1980) with step-size control,
 *                         one of the further Runge-Kutta methods the paper's
 *                         conclusions name.  The first trial step is dl (or
 *                         dl_r_scale r_0 when dl = 0); when dl_r_scale > 0
 *                         every step is at most dl_r_scale r (r at its start).
 *                         An attempt is accepted when the RMS over the 8
 *                         state components of e_i / (atol + rtol max(|y_i|,
 *                         |y5_i|)) is <= 1 (e = fifth- minus fourth-order
 *                         result); the next step is h 2^(j/4) with
 *                         j = floor(4 log2 0.9 - 0.8 log2 err) (0.9 err^-1/5
 *                         taken down to a grid, so that the rounding noise
 *                         of the error estimate does not reach the step
 *                         sizes), j in [-10, 13], j <= 0 right after a
 *                         rejection and j <= -1 after one.
 *                         n_steps_cap, the reported steps and the trajectory
 *                         stride count attempts; capture and non-finite are
 *                         tested on every attempt (at its result and its
 *                         stage points, as for RK4), escape on accepted
 *                         steps.  Any form (in the canonical forms p_t and
 *                         p_ph stay exactly constant, as with RK4).  Requires
 *                         atol > 0 and rtol >= 0.  Every entry point
 *                         (bundles and servers as for the forms), in both
 *                         precisions, except malbec_trace_noalloc, which
 *                         takes it in FP64 only.  MALBEC_FP32_MIXED: attempts in FP32
 *                         on the compensated state, in FP64 in the FP64
 *                         zones, the error norm and the step rule in the
 *                         precision of the attempt; requires rtol >=
 *                         MALBEC_DOPRI5_MIXED_RTOL_MIN (an FP32 error
 *                         estimate carries rounding noise of ~1e-7 of the
 *                         state; MALBEC_EINVAL below it).  The block ray
 *                         exchange is off for this method (a ray keeps its
 *                         lane and its step-size state).
 * rtol, atol: the tolerances of MALBEC_METHOD_DOPRI5 (ignored by RK4). */
#define MALBEC_FORM_GEODESIC 0
#define MALBEC_FORM_HAMILTONIAN 1
#define MALBEC_FORM_ADM 2
#define MALBEC_METHOD_RK4 0
#define MALBEC_METHOD_DOPRI5 1
/* smallest rtol of MALBEC_METHOD_DOPRI5 in MALBEC_FP32_MIXED */
#define MALBEC_DOPRI5_MIXED_RTOL_MIN 1e-6
typedef struct {
  double eps_hor;
  double r_esc;
  uint32_t n_steps_cap;
  double dl;
  double dl_r_scale;
  uint32_t form;
  uint32_t method;
  double rtol;
  double atol;
} malbec_term;

typedef enum {
  MALBEC_OUT_FINAL = 0,   /* final state, lambda, invariants, steps, fate */
  MALBEC_OUT_STRIDED = 1, /* FINAL plus a trajectory sample every `stride` steps */
  MALBEC_OUT_STRIDED_CARTESIAN = 2 /* FINAL plus a sample (t, x, y, z) every `stride` steps:
                                      the paper's output records (Sec. 5), with
                                      x = sqrt(r^2 + a^2) sin th cos ph,
                                      y = sqrt(r^2 + a^2) sin th sin ph, z = r cos th
                                      (Sec. 2 eq. coord) */
} malbec_out_mode;

typedef enum {
  MALBEC_FP64 = 0,      /* every operation in double precision */
  MALBEC_FP32_MIXED = 1 /* FP32 RHS and stages, compensated (hi, lo) FP32 state,
                           FP64 steps inside the FP64 zone, FP64 lambda and invariants */
} malbec_precision;

/* FP32_MIXED FP64 zone: a step runs in FP64 when, at its start,
 *   r < MALBEC_ZONE_HORIZON_FACTOR * r_+                      (every ray), or
 *   r < r_ph,retro(a) + MALBEC_ZONE_PHOTON_MARGIN * M        (null rays), or
 *   |sin theta| < MALBEC_ZONE_POLE_SIN   (timelike rays near the polar axis,
 *                                         where the BL Christoffel symbols
 *                                         diverge: keeps E, L_z, Q drift
 *                                         below 1e-6; null rays that come
 *                                         this close are ill-conditioned in
 *                                         any precision),
 * r_ph,retro = 2M (1 + cos(2/3 arccos(a/M))) the retrograde circular photon
 * orbit, the outer edge of the spherical photon orbits.  A ray is null when
 * |g(u,u)| <= 1e-6 (u^t)^2 |g_tt| at its start. */
#define MALBEC_ZONE_HORIZON_FACTOR 2.0
#define MALBEC_ZONE_PHOTON_MARGIN 0.5
#define MALBEC_ZONE_POLE_SIN 0.2

/* The FP64 zone in force for subsequent FP32_MIXED calls of this process
 * (the defaults above until changed).  Larger zones trade speed for accuracy.
 * Requires horizon_factor >= 1, photon_margin >= 0, 0 <= pole_sin <= 1;
 * NULL restores the defaults.  Thread-safe; calls already enqueued keep the
 * zone they were given. */
typedef struct {
  double horizon_factor;
  double photon_margin;
  double pole_sin;
} malbec_mixed_zone;

int malbec_set_mixed_zone(const malbec_mixed_zone* zone);
int malbec_get_mixed_zone(malbec_mixed_zone* zone);

/* Launch configuration of the persistent trace kernels (process-wide, for
 * subsequent calls; a 0 field keeps the automatic choice):
 *   threads_per_block  32..256, a multiple of 32 (automatic: 128, or 32 for
 *                      batches smaller than 4 warps per SM);
 *   blocks_per_sm      resident blocks per SM, capped by occupancy
 *                      (automatic: 8 warps per SM for FP64 -- two per SM
 *                      sub-partition keep the FP64 unit busy --, 8 for
 *                      FP32_MIXED, 12 for FP32_MIXED whole-image cameras);
 *   refill_min         a warp takes new rays once this many lanes are idle
 *                      (automatic: 2 for FP64; for FP32_MIXED whole-image
 *                      cameras 32, 8 or 1 for >= 16, >= 4 or fewer rays per
 *                      resident lane -- neighbouring pixels taken together
 *                      take their FP64 zone steps together --, and 1 for
 *                      other FP32_MIXED sources);
 *   zone_batch         FP32_MIXED: an FP64-zone warp step waits for this many
 *                      lanes (automatic: 8 with the exchange below, 32
 *                      without) ...
 *   zone_wait          ... or until a waiting lane sat out this many warp
 *                      steps (automatic: 1 for whole-image cameras, 64
 *                      otherwise);
 *   exchange           FP32_MIXED: 1 = the warps of a block hand FP64-zone
 *                      rays to one zone warp per block and take FP32 rays
 *                      back (zone steps run with fuller warps), 2 = every
 *                      ray stays in its warp (automatic: 2 for whole-image
 *                      cameras, whose rays spend few steps in the zone, 1
 *                      otherwise; always 2 for MALBEC_METHOD_DOPRI5);
 *   zone_wait_limit_us with the exchange, the longest a block's zone warp,
 *                      once it has no ray left, waits for the other warps of
 *                      its block before it closes its bank and leaves (the
 *                      others then take their FP64-zone steps in place);
 *                      measured on the device clock from the moment the zone
 *                      warp ran out of work (automatic: 2 s).  A wait that
 *                      runs out is counted: see malbec_wait_status.
 * The choice changes speed only: every ray's arithmetic is the same.
 * NULL restores all-automatic.  Thread-safe. */
typedef struct {
  uint32_t threads_per_block;
  uint32_t blocks_per_sm;
  uint32_t refill_min;
  uint32_t zone_batch;
  uint32_t zone_wait;
  uint32_t exchange;
  uint32_t zone_wait_limit_us;
} malbec_launch_config;

int malbec_set_launch_config(const malbec_launch_config* cfg);
int malbec_get_launch_config(malbec_launch_config* cfg);

/* ---------------------------------------------------------------- output layout */
/* Offsets (bytes from the start of `out`) of the output fields of
 * malbec_trace.  Every field starts on a 256-byte boundary.
 *   y       double[8][n]     final state (SoA)
 *   lambda  double[n]        affine parameter (sum of the steps taken)
 *   inv0    double[4][n]     E = -p_t, L_z = p_phi, Carter Q, norm g(u,u) at the start
 *   inv1    double[4][n]     the same at the end (always FP64)
 *   steps   uint32[n]        RK4 steps taken
 *   fate    uint8[n]         MALBEC_FATE_*, with MALBEC_FATE_DRIFTED or-ed in when set
 *   traj    STRIDED modes only: per ray `n_samples` samples of C components
 *           (C = 8, the state, for MALBEC_OUT_STRIDED; C = 4, (t, x, y, z),
 *           for MALBEC_OUT_STRIDED_CARTESIAN), ray-major:
 *           traj[(i * n_samples + k) * C + c]; double for FP64, float for
 *           FP32_MIXED (the hi word of the state, or (t, x, y, z) from it).
 *           Sample k is taken after k * stride steps (sample 0 = initial
 *           state); samples after the ray terminated are NaN.
 *           n_samples = n_steps_cap / stride + 1. */
typedef struct {
  size_t y, lambda, inv0, inv1, steps, fate, traj;
  uint64_t n_samples;
  size_t total; /* bytes to allocate for `out` */
} malbec_layout;

int malbec_out_layout(malbec_out_mode mode, malbec_precision prec, uint64_t n,
                      uint32_t n_steps_cap, uint32_t stride, malbec_layout* layout);
/* = layout.total, or 0 on invalid arguments. */
size_t malbec_out_bytes(malbec_out_mode mode, malbec_precision prec, uint64_t n,
                        uint32_t n_steps_cap, uint32_t stride);

/* ---------------------------------------------------------------- tracing */
/* Integrate n rays from the initial states `ics` (device, double[8][n] SoA)
 * until each terminates (see fates).  The right-hand side is the one of
 * term.form: by default the geodesic equation du^mu/dl = -Gamma^mu_ab u^a u^b
 * (the second-order form of the canonical equations, Sec. 2 eq. Ham)
 * specialised for Schwarzschild or Kerr; the integrator is term.method's
 * (by default the classical 4-stage RK4).  Rays are pulled from
 * a device work queue by persistent warps, and a lane whose ray ends takes
 * the next one, so uneven step counts do not idle lanes.
 * out: device, layout.total bytes (malbec_out_layout), caller-owned.
 * Validation (MALBEC_EINVAL): M > 0, 0 <= a < M, finite step > 0,
 * r_esc > capture radius, stride > 0 in STRIDED mode, n > 0, non-NULL
 * pointers.  Initial radii are not read on the host; a ray starting inside
 * the capture radius ends CAPTURED after one step.
 * Scratch: a 256-byte work-queue block is taken from the stream-ordered
 * allocator (cudaMallocAsync / cudaFreeAsync on `stream`). */
int malbec_trace(malbec_metric m, const double* ics, uint64_t n, malbec_term t,
                 malbec_out_mode mode, uint32_t stride, malbec_precision prec, void* out,
                 malbec_stream stream);

/* malbec_trace for callers that cannot allocate device memory.  (The paper
 * has no counterpart: this is a property of the library, not of the method.)
 * Who needs it: code that records work into a CUDA graph under a capture mode
 * that forbids allocation calls, real-time loops that must never enter the
 * allocator (an allocation may synchronise or grow a memory pool at an
 * unpredictable moment), and embedders that hand out every byte of device
 * memory from their own arena and do not let libraries call cudaMalloc.
 * Same arguments, validation, results and errors as malbec_trace, but the
 * 256-byte work-queue block lives in a static __device__ array of
 * MALBEC_NOALLOC_SCRATCH_BYTES bytes inside libmalbec.so, held by every GPU
 * that loads the library until the process exits.  No cudaMalloc, cudaFree,
 * stream-ordered or library allocation is made: the call enqueues a memset of
 * the block (it keeps the previous call's contents) and the kernel.
 *  - The first call in a CUDA context (in practice the first call on each
 *    device, with that device current) looks up the array's device address
 *    (cudaGetSymbolAddress) and caches it under the context's id; a context
 *    made after cudaDeviceReset looks it up again.  Make that first call
 *    before any stream capture.
 *  - Every call on a device shares the one array: calls whose work overlaps
 *    on the GPU (different streams, or graphs replayed concurrently) race on
 *    the work queue and give wrong results.  Serialise them.
 *  - A trace needs one 256-byte block whatever n is, so this call never
 *    returns MALBEC_ESCRATCH (the code is kept for entry points whose
 *    scratch grows with their arguments).
 *  - The buffers are not checked on the host beyond NULL and alignment (the
 *    library sees raw pointers): ics must hold 8 n doubles, a_per_ray n
 *    doubles, out layout.total bytes, all on the current device. */
#define MALBEC_NOALLOC_SCRATCH_BYTES 256
int malbec_trace_noalloc(malbec_metric m, const double* ics, uint64_t n, malbec_term t,
                         malbec_out_mode mode, uint32_t stride, malbec_precision prec, void* out,
                         malbec_stream stream);

/* ---------------------------------------------------------------- camera */
/* Backward null-ray camera (not in the paper; Bardeen 1973 impact
 * parameters).  Pixel p = j * nx + i has impact parameters
 *   alpha = -fov_half + 2 fov_half (i + 1/2)/nx,  beta = -fov_half + 2 fov_half (j + 1/2)/ny.
 * The arriving photon has E = 1, L_z = -alpha sin(incl),
 * Q = beta^2 + cos^2(incl)(alpha^2 - a^2), p_theta = sign(beta) sqrt(Theta(incl)),
 * p_r = +sqrt(R(r_obs))/Delta(r_obs), observer at (t, r, theta, phi) =
 * (0, r_obs, incl, 0).  The ray is traced backward by integrating forward in
 * lambda with p reversed; u = g^{-1}(-p).  Initial states are built in the
 * kernel (no input array). */
typedef struct {
  double r_obs; /* observer radius, > capture radius and < r_esc */
  double incl;  /* observer inclination (radians), in (0, pi) */
  double fov_half;
  uint32_t nx, ny;
} malbec_camera;

/* Camera output offsets (bytes, 256-aligned): fate uint8[n], steps uint32[n],
 * theta double[n], phi double[n] (final theta and unwrapped phi of each
 * ray), n = nx * ny. */
typedef struct {
  size_t fate, steps, theta, phi;
  size_t total;
} malbec_camera_layout;

int malbec_camera_out_layout(const malbec_camera* cam, malbec_camera_layout* layout);

/* Render one camera image: trace every pixel's ray.  m.a_per_ray must be
 * NULL.  out: device, layout.total bytes.  Rays are started centre columns
 * first (smallest |alpha|, i.e. smallest |L_z|: the rays that pass closest to
 * the polar axis and take the most steps); the order is a schedule only, every
 * pixel's output is the same as in any other order. */
int malbec_trace_camera(malbec_metric m, const malbec_camera* cam, malbec_term t,
                        malbec_precision prec, void* out, malbec_stream stream);

/* Initial states of the camera pixels `pixels` (device uint64[n] pixel
 * indices) into ics (device double[8][n]); the same construction the camera
 * kernel uses. */
int malbec_ic_camera(malbec_metric m, const malbec_camera* cam, const uint64_t* pixels,
                     uint64_t n, double* ics, malbec_stream stream);

/* ---------------------------------------------------------------- uneven bundles */
/* Many independent bundles of rays, each with its own black hole, kind, step
 * rule, step cap and output buffer, traced by ONE persistent work-queue
 * launch (not in the paper, whose runs trace one set of initial conditions
 * at a time).  Warps take rays bundle by bundle, the costliest bundles first
 * (estimated cost n * cap for orbits, n * min(cap, 300) for camera rays), so
 * bundles whose rays end after very different step counts keep every lane
 * busy. */
#define MALBEC_BUNDLE_STATES 0 /* rays from `ics` (device double[8][n]) */
#define MALBEC_BUNDLE_CAMERA 1 /* backward camera pixels 0..n-1 (n <= nx * ny) */
#define MALBEC_BUNDLE_BOUND 2  /* generic bound orbits of malbec_ic_bound with
                                  the spin fixed at `a`, particles 0..n-1 of `seed` */
typedef struct {
  int32_t kind;
  uint32_t n;          /* rays, >= 1 */
  double M, a;         /* M > 0, 0 <= a < M */
  malbec_term term;
  malbec_camera camera; /* CAMERA only */
  const double* ics;    /* STATES only */
  uint64_t seed;        /* BOUND only */
  void* out;            /* device, 256-byte aligned, malbec_bundle_out_bytes() bytes */
} malbec_bundle;

/* Output of one bundle: STATES and BOUND use the FINAL layout of
 * malbec_out_layout(MALBEC_OUT_FINAL, prec, n, cap, 0); CAMERA the camera
 * layout of an n x 1 camera (fate, steps, theta, phi of n pixels). */
size_t malbec_bundle_out_bytes(const malbec_bundle* b, malbec_precision prec);

/* Trace `count` bundles (host array) in one launch on `stream` -- one
 * persistent launch per class of (term.form, term.method) present, one after
 * the other, each kernel specialised for its class (a table of one class, the
 * usual case, is one launch).  Every bundle is validated as malbec_trace /
 * malbec_trace_camera would (MALBEC_EINVAL before anything is enqueued).
 * Scratch (job table, counters) comes from the stream-ordered allocator. */
int malbec_trace_bundles(const malbec_bundle* bundles, uint32_t count, malbec_precision prec,
                         malbec_stream stream);

/* A plan: the bundles uploaded once and their launch recorded as a CUDA
 * graph (reset of the work-queue counters + the persistent kernel), replayed
 * by malbec_plan_launch with a single cudaGraphLaunch.  The plan owns its
 * device table (cudaMalloc at creation); the bundles' `ics` and `out`
 * buffers must stay valid while it is used.  Plans take the launch
 * configuration in force at creation, or the one malbec_plan_autotune picks:
 * it replays the plan under candidate configurations (block size, blocks per
 * SM, refill granularity, FP64-zone batching, block ray exchange) on
 * `stream`, blocking the caller -- each once after a warm-up replay, the three
 * fastest twice more -- and keeps the one with the best replay (written to
 * `best` if non-NULL). */
typedef struct malbec_plan malbec_plan;
int malbec_plan_create(const malbec_bundle* bundles, uint32_t count, malbec_precision prec,
                       malbec_plan** plan);
int malbec_plan_launch(malbec_plan* plan, malbec_stream stream);
int malbec_plan_autotune(malbec_plan* plan, malbec_stream stream, malbec_launch_config* best);
int malbec_plan_destroy(malbec_plan* plan);

/* ---------------------------------------------------------------- serving */
/* A request loop with continuous batching (not in the paper).  Jobs are
 * bundles (malbec_bundle without `out`: the server allocates each job's
 * output from its HBM budget).  One resident trace kernel serves every
 * admitted job at once: idle lanes take rays from the active jobs,
 * smallest estimated job first, so a request that arrives while others run
 * starts as soon as lanes free up and its rays overlap with theirs on the
 * device.  A ray's result does not depend on which other jobs ran with it.
 *  - Admission: a job is admitted when the active set has a free place
 *    (max_active) and its output fits in hbm_budget minus the bytes held by
 *    admitted, not yet released jobs; otherwise it waits in a FIFO of at most
 *    max_pending jobs (malbec_submit returns MALBEC_EBUSY when that is full).
 *  - The kernel leaves by itself once every one of its warps has been
 *    without work for idle_timeout_s (measured on the device clock; the
 *    whole grid leaves at once, so a job never runs on a partly exited
 *    kernel), and is relaunched by the next submit or poll that finds work.
 *    Job slots form a ring of 65536 descriptors.
 *  - Completion is signalled by the device in mapped host memory; polling
 *    never synchronises the device.
 * All calls are thread-safe.  malbec_server_destroy waits for running rays
 * to finish (new rays are no longer started) and frees everything. */
typedef struct malbec_server malbec_server;
typedef struct {
  size_t hbm_budget;      /* bytes for job outputs (e.g. 150e9) */
  uint32_t max_active;    /* jobs served at once, 1..4096 */
  uint32_t max_pending;   /* queued jobs beyond that, >= 1 */
  malbec_precision precision;
  double idle_timeout_s;  /* kernel exit after this long without work, > 0 */
  uint32_t form;          /* MALBEC_FORM_* of every job of this server (0: geodesic) */
  uint32_t method;        /* MALBEC_METHOD_* of every job (0: RK4) */
} malbec_server_config;

typedef struct {
  uint64_t submitted, admitted, completed, released;
  uint64_t pending, active;
  uint64_t bytes_in_use;
  uint64_t kernel_launches;
} malbec_server_stats;

int malbec_server_create(const malbec_server_config* cfg, malbec_server** server);
int malbec_server_destroy(malbec_server* server);
/* Non-blocking.  `job->out` is ignored.  STATES jobs read `ics` while they
 * run: keep it valid until the job is done.  job->term.form and
 * job->term.method must be the server's (MALBEC_EINVAL otherwise): one server
 * runs one class of equations and integrator, its resident kernel
 * specialised for it; each job keeps its own tolerances. */
int malbec_submit(malbec_server* server, const malbec_bundle* job, uint64_t* job_id);
/* Non-blocking: *done = 1 once every ray of the job has finished. */
int malbec_poll(malbec_server* server, uint64_t job_id, int* done);
/* Device pointer and size of a finished job's output (bundle layout); valid
 * until malbec_job_release.  MALBEC_EBUSY while the job runs. */
int malbec_job_output(malbec_server* server, uint64_t job_id, void** out, size_t* bytes);
/* Copy a finished job's output (all `bytes` of it) to `dst` (device or
 * pinned host memory) on `stream`.  MALBEC_EBUSY while the job runs. */
int malbec_job_copy_output(malbec_server* server, uint64_t job_id, void* dst, size_t bytes,
                           malbec_stream stream);
/* Give the job's memory back to the budget (after its output was read). */
int malbec_job_release(malbec_server* server, uint64_t job_id);
int malbec_server_stats_get(malbec_server* server, malbec_server_stats* stats);

/* ---------------------------------------------------------------- initial data */
/* Circular equatorial timelike orbits at the radii `radii` (device double[n]):
 * Schwarzschild E, L from Sec. 4 eqs. COrbit/COrbit2 when a = 0, Bardeen's
 * prograde (prograde != 0) or retrograde E, L otherwise; state
 * x = (0, r, pi/2, 0), u = g^{-1}(-E, 0, 0, L).  ics: device double[8][n].
 * Radii where no circular orbit exists give NaN states. */
int malbec_ic_circular(malbec_metric m, const double* radii, uint64_t n, int prograde,
                       double* ics, malbec_stream stream);

/* Generic bound Kerr orbits (not in the paper).  Particle i draws with the
 * SplitMix64 counter-based generator (seed, counter i*256 + k):
 *   a = a_max U (counter i*256), unless spin_fixed (then a = a_max);
 *   candidates j = 0..63: r_p = r_lo + (10M - r_lo) U(i*256+4j+1) with
 *   r_lo = ISCO_prograde(a) + 0.5M, e = 0.7 U(i*256+4j+2), iota = pi U(i*256+4j+3);
 * and keeps the first candidate that is bound and stable: (E, L_z, Q) solve
 * R(r_p) = R(r_a) = 0 (R(r_p) = R'(r_p) = 0 when e < 1e-6), r_a = r_p (1+e)/(1-e),
 * cos iota = L_z / sqrt(L_z^2 + Q), 0 < E < 1, third root of R below r_p.
 * State: x = (0, r_p, pi/2, 0), p = (-E, 0, +sqrt(Q), L_z), u = g^{-1} p.
 * If all 64 candidates fail, the prograde circular equatorial orbit at 10M.
 * Outputs (device): ics double[8][n], spins double[n], accepted int32[n]
 * (candidate index, -1 for the fallback); particle indices run from
 * index0 to index0 + n - 1. */
int malbec_ic_bound(double M, double a_max, int spin_fixed, uint64_t seed, uint64_t index0,
                    uint64_t n, double* ics, double* spins, int32_t* accepted,
                    malbec_stream stream);

/* The paper's initial-condition rows (Sec. 5: columns t, r, theta, phi, p_t,
 * p_r, p_theta, p_phi, where the p_t column holds E > 0) to states: with
 * p = (-E, p_r, p_theta, p_phi), x is copied and u = g^{-1} p (eq. kerr),
 * per-ray spins from m.a_per_ray if given.  rows and ics: device
 * double[8][n] (SoA, the transpose of the paper's row layout), distinct
 * buffers; MALBEC_EINVAL for a bad metric, n = 0, NULL or aliased buffers. */
int malbec_ic_from_paper(malbec_metric m, const double* rows, uint64_t n, double* ics, malbec_stream stream);

/* E, L_z, Q (Carter), norm g(u,u) of n states (device double[8][n]) into
 * inv (device double[4][n]), in FP64. */
int malbec_invariants(malbec_metric m, const double* states, uint64_t n, double* inv,
                      malbec_stream stream);

/* ---------------------------------------------------------------- measurement */
/* Measured non-tensor FMA throughput of the current device: FP64
 * (precision = MALBEC_FP64) or FP32 (MALBEC_FP32_MIXED) dependent-chain-free
 * FMA loop, all SMs, timed with CUDA events.  Blocks the calling thread.
 * Writes GFLOP/s (2 flops per FMA). */
int malbec_measure_fma_peak(malbec_precision prec, double* gflops);

/* The bare FP64 RK4 step loop of one form (MALBEC_FORM_*): the step the trace
 * kernels take (same right-hand side, Sec. 2 eq. kerr with eq. geo, eq. Ham
 * or eq. ADM, and the classical RK4 tableau), with no work queue, termination
 * test or output: every thread follows an inclined bound orbit of Kerr
 * a = 0.9 M near r = 10 M with dtau = 0.5 for 4000 steps, two warps per SM
 * sub-partition (the FP64 trace kernels' shape), all SMs.  Blocks the calling thread; best of three launches.
 * Writes RK4 steps/s: the ceiling of a trace kernel for that right-hand
 * side's instruction mix.  MALBEC_EINVAL for another form. */
int malbec_measure_step_loop(uint32_t form, double* steps_per_s);

/* Self-check of three FP64 device helpers of the right-hand sides, on 2^22
 * seeded samples: the stage sine/cosine by angle addition (|d| <= 1/4)
 * against CUDA's sincos at the same, exactly representable angle, the
 * refined reciprocal against the IEEE division 1.0 / x (x in 2^[-60, 60]),
 * and the steps' own sine/cosine (Cody-Waite reduction and Taylor series)
 * against CUDA's sincos on x in [-4, 8], next to the multiples of pi/2
 * there, and up to 2^30 in magnitude.  err[0], err[1]: max absolute stage sine, cosine difference;
 * err[2]: max reciprocal difference in units of the last place of 1/x;
 * err[3]: max relative error of the hardware reciprocal estimate before
 * refinement; err[4], err[5]: max absolute sine, cosine difference of the
 * steps' sine/cosine.  Blocks the calling thread. */
int malbec_check_fp64_helpers(double err[6]);

/* Self-check of the operand forms the kernels compute in (not in the paper),
 * bit for bit on 2^22 seeded samples of every class of value (zeros,
 * subnormals, normals, infinities, NaN; a NaN matches a NaN): counts[0..2]:
 * mismatches of the FP64 forms fma(x, y, -0), fma(x, 1, y), fma(x, 1, -y)
 * (constants in per-thread registers) against x*y, x + y, x - y; counts[3]:
 * of the exponent doubling against x + x (finite normal x); counts[4..6]: of
 * the paired FP32 add, subtract, and multiply and fma against the scalar
 * operations; counts[7]: of the paired compensated update against the scalar
 * one.  MALBEC_EINVAL for a null pointer.  Blocks the calling thread. */
int malbec_check_operand_forms(uint64_t counts[8]);

/* Bounded device-side waits (not in the paper).  The one wait a trace
 * kernel makes on other warps is the zone warp's wait for the rest of its
 * block (launch configuration, zone_wait_limit_us); when it runs out the
 * zone warp leaves, the other warps take their FP64-zone steps in place, and
 * results are unchanged.  Every expiry on the current device increments a
 * device-wide counter.  This call waits for the current device's work
 * (cudaDeviceSynchronize), writes the counter's total to *timeouts (if not
 * NULL), and returns MALBEC_ETIMEDOUT if the total grew since the previous
 * call in this process, MALBEC_OK otherwise. */
int malbec_wait_status(uint64_t* timeouts);

/* Library build information (static string). */
const char* malbec_build_info(void);

#ifdef __cplusplus
}
#endif
#endif

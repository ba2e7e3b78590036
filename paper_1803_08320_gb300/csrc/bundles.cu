// bundles.cu -- uneven bundles of rays in one persistent launch (host side):
// validation, the device job table, the costliest-first job order, the
// one-shot entry point, and plans (table uploaded once, launch recorded as a
// CUDA graph, launch configuration autotuned by replay).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.h"

namespace malbec {
namespace {

size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

struct CameraFields {
  size_t fate, steps, theta, phi, total;
};

CameraFields camera_fields(uint64_t n) {
  CameraFields f;
  size_t off = 0;
  f.fate = off;
  off = align256(off + n);
  f.steps = off;
  off = align256(off + n * sizeof(uint32_t));
  f.theta = off;
  off = align256(off + n * sizeof(double));
  f.phi = off;
  off = align256(off + n * sizeof(double));
  f.total = off;
  return f;
}

int validate(const malbec_bundle& b, malbec_precision prec) {
  if (b.n == 0 || !b.out || ((uintptr_t)b.out & 255u) != 0) return MALBEC_EINVAL;
  const malbec_metric m = {b.M, b.a, nullptr};
  int rc = check_metric(m);
  if (rc) return rc;
  rc = check_term(b.term, m);  // form and method included
  if (rc) return rc;
  rc = check_method_precision(b.term, prec, true);
  if (rc) return rc;
  if (b.kind == MALBEC_BUNDLE_CAMERA) {
    rc = check_camera_desc(m, &b.camera, &b.term);
    if (rc) return rc;
    if ((uint64_t)b.n > (uint64_t)b.camera.nx * b.camera.ny) return MALBEC_EINVAL;
  } else if (b.kind == MALBEC_BUNDLE_STATES) {
    if (!b.ics) return MALBEC_EINVAL;
  } else if (b.kind != MALBEC_BUNDLE_BOUND) {
    return MALBEC_EINVAL;
  }
  if (prec != MALBEC_FP64 && prec != MALBEC_FP32_MIXED) return MALBEC_EINVAL;
  return MALBEC_OK;
}

}  // namespace

int validate_job(const malbec_bundle& b, malbec_precision prec) {
  malbec_bundle c = b;
  c.out = reinterpret_cast<void*>(256);  // the server allocates the output
  return validate(c, prec);
}

void fill_job_desc(const malbec_bundle& b, malbec_precision prec, void* out, uint64_t job_id, JobDesc* J,
                   double* cost) {
  memset(J, 0, sizeof(*J));
  J->kind = b.kind;
  J->cap = b.term.n_steps_cap;
  J->n = b.n;
  J->job_id = job_id;
  J->M = b.M;
  J->a = b.a;
  J->eps_hor = b.term.eps_hor;
  J->r_esc = b.term.r_esc;
  J->dl = b.term.dl;
  J->dl_r_scale = b.term.dl_r_scale;
  J->seed = b.seed;
  J->form = b.term.form;
  J->method = b.term.method;
  J->rtol = b.term.rtol;
  J->atol = b.term.atol;
  J->ics = b.ics;
  char* o = static_cast<char*>(out);
  if (b.kind == MALBEC_BUNDLE_CAMERA) {
    J->cam = make_camera_const(b.M, b.a, b.camera);
    const CameraFields f = camera_fields(b.n);
    J->fate_out = reinterpret_cast<uint8_t*>(o + f.fate);
    J->steps_out = reinterpret_cast<uint32_t*>(o + f.steps);
    J->theta_out = reinterpret_cast<double*>(o + f.theta);
    J->phi_out = reinterpret_cast<double*>(o + f.phi);
    *cost = (double)b.n * std::min<double>(b.term.n_steps_cap, 300.0);
  } else {
    malbec_layout L;
    malbec_out_layout(MALBEC_OUT_FINAL, prec, b.n, b.term.n_steps_cap, 0, &L);
    J->y_out = reinterpret_cast<double*>(o + L.y);
    J->lambda_out = reinterpret_cast<double*>(o + L.lambda);
    J->inv0_out = reinterpret_cast<double*>(o + L.inv0);
    J->inv1_out = reinterpret_cast<double*>(o + L.inv1);
    J->steps_out = reinterpret_cast<uint32_t*>(o + L.steps);
    J->fate_out = reinterpret_cast<uint8_t*>(o + L.fate);
    *cost = (double)b.n * (double)b.term.n_steps_cap;
  }
}

namespace {

// The class of a job: its (form, method); one persistent launch runs the jobs
// of one class (the kernel is specialised for its equations and integrator).
uint32_t job_class(const JobDesc& J) { return J.form * 2u + J.method; }

// A class's run of the order array: jobs order[first .. first + count - 1].
struct ClassRun {
  uint32_t form, method, first, count;
  uint64_t rays;
};

int build_jobs(const malbec_bundle* bundles, uint32_t count, malbec_precision prec, std::vector<JobDesc>& jobs,
               std::vector<uint32_t>& order, std::vector<ClassRun>& runs, uint64_t* total_rays) {
  if (!bundles || count == 0) return MALBEC_EINVAL;
  jobs.assign(count, JobDesc());
  uint64_t total = 0;
  std::vector<double> cost(count);
  for (uint32_t i = 0; i < count; ++i) {
    const malbec_bundle& b = bundles[i];
    int rc = validate(b, prec);
    if (rc) return rc;
    fill_job_desc(b, prec, b.out, 0, &jobs[i], &cost[i]);
    total += b.n;
  }
  // jobs grouped by class (form, method), costliest first within a class
  order.resize(count);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    const uint32_t cx = job_class(jobs[x]), cy = job_class(jobs[y]);
    return cx != cy ? cx < cy : cost[x] > cost[y];
  });
  runs.clear();
  for (uint32_t k = 0; k < count; ++k) {
    const JobDesc& J = jobs[order[k]];
    if (runs.empty() || job_class(jobs[order[runs.back().first]]) != job_class(J))
      runs.push_back(ClassRun{J.form, J.method, k, 0u, 0ull});
    runs.back().count++;
    runs.back().rays += J.n;
  }
  *total_rays = total;
  return MALBEC_OK;
}

// Scratch block: [jobs][order][counters][cursors], each 256-aligned; the
// counters and the cursors (one per class run; the tail from `ctr` on) are
// zeroed before a launch.
constexpr uint32_t kMaxRuns = 8;  // classes: 3 forms x 2 methods
struct BlockLayout {
  size_t jobs, ctr, order, cursor, total;
};
BlockLayout block_layout(uint32_t count) {
  BlockLayout b;
  size_t off = 0;
  b.jobs = off;
  off = align256(off + count * sizeof(JobDesc));
  b.order = off;
  off = align256(off + count * sizeof(uint32_t));
  b.ctr = off;
  off = align256(off + count * sizeof(JobCounter));
  b.cursor = off;
  off = align256(off + kMaxRuns * sizeof(unsigned int));
  b.total = off;
  return b;
}

// Parameters of the launch of class run `k`: its slice of the order array,
// its own cursor, its equations and integrator.
void fill_params(TraceParams& p, char* block, const BlockLayout& bl, const ClassRun& run, uint32_t k) {
  memset(&p, 0, sizeof(p));
  p.M = 1.0;
  p.n = run.rays;
  p.stride = 1;
  p.form = run.form;
  p.method = run.method;
  p.jobs = reinterpret_cast<const JobDesc*>(block + bl.jobs);
  p.job_ctr = reinterpret_cast<JobCounter*>(block + bl.ctr);
  p.job_order = reinterpret_cast<const uint32_t*>(block + bl.order) + run.first;
  p.n_jobs = run.count;
  p.job_cursor = reinterpret_cast<unsigned int*>(block + bl.cursor) + k;
  fill_zone(p);
}

// Enqueue the launches of every class run on `s` (after the counters and
// cursors have been zeroed): one persistent launch per class, in class order.
int launch_runs(char* block, const BlockLayout& bl, const std::vector<ClassRun>& runs, bool mixed,
                const malbec_launch_config* cfg, cudaStream_t s, cudaError_t* err) {
  *err = cudaSuccess;
  for (uint32_t k = 0; k < (uint32_t)runs.size(); ++k) {
    TraceParams p;
    fill_params(p, block, bl, runs[k], k);
    LaunchShape shape;
    int refill_min = 1;
    int rc = cfg ? choose_shape_cfg(true, mixed, kSrcJobs, kSinkJobs, runs[k].rays, *cfg, &shape, &refill_min)
                 : choose_shape(true, mixed, kSrcJobs, kSinkJobs, runs[k].rays, &shape, &refill_min);
    if (rc) return rc;
    p.refill_min = refill_min;
    if (cfg) {
      if (cfg->zone_batch) p.zone_batch = (int)cfg->zone_batch;
      if (cfg->zone_wait) p.zone_wait = (int)cfg->zone_wait;
      if (cfg->exchange) p.exchange = cfg->exchange == 1 ? 1 : 0;
      if (cfg->zone_wait_limit_us) p.zone_wait_ns = (uint64_t)cfg->zone_wait_limit_us * 1000ull;
    }
    *err = launch_trace(p, true, mixed, kSrcJobs, kSinkJobs, shape, s);
    if (*err != cudaSuccess) return MALBEC_OK;
  }
  return MALBEC_OK;
}

}  // namespace
}  // namespace malbec

using namespace malbec;

struct malbec_plan {
  int device = 0;
  uint32_t count = 0;
  uint64_t total_rays = 0;
  bool mixed = false;
  void* block = nullptr;
  BlockLayout bl;
  std::vector<ClassRun> runs;
  malbec_launch_config cfg = {0, 0, 0, 0, 0, 0, 0};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// Record [zero the counters and the cursor] + [the persistent kernel] with
// launch configuration `cfg` as the plan's graph.
int record_plan(malbec_plan* P, const malbec_launch_config& cfg) {
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return set_cuda_error(e);
  cudaGraph_t g = nullptr;
  int rc = MALBEC_OK;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    char* blk = static_cast<char*>(P->block);
    cudaError_t e1 = cudaMemsetAsync(blk + P->bl.ctr, 0, P->bl.total - P->bl.ctr, s);
    cudaError_t e2 = e1;
    if (e1 == cudaSuccess) rc = launch_runs(blk, P->bl, P->runs, P->mixed, &cfg, s, &e2);
    e = cudaStreamEndCapture(s, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  cudaStreamDestroy(s);
  if (rc != MALBEC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != MALBEC_OK ? rc : set_cuda_error(e);
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return set_cuda_error(e);
  }
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->graph = g;
  P->exec = x;
  P->cfg = cfg;
  return MALBEC_OK;
}

}  // namespace

extern "C" {

size_t malbec_bundle_out_bytes(const malbec_bundle* b, malbec_precision prec) {
  if (!b || b->n == 0) return 0;
  if (b->kind == MALBEC_BUNDLE_CAMERA) return camera_fields(b->n).total;
  return malbec_out_bytes(MALBEC_OUT_FINAL, prec, b->n, b->term.n_steps_cap, 0);
}

int malbec_trace_bundles(const malbec_bundle* bundles, uint32_t count, malbec_precision prec, malbec_stream stream) {
  std::vector<JobDesc> jobs;
  std::vector<uint32_t> order;
  std::vector<ClassRun> runs;
  uint64_t total = 0;
  int rc = build_jobs(bundles, count, prec, jobs, order, runs, &total);
  if (rc) return rc;
  const bool mixed = prec == MALBEC_FP32_MIXED;
  const BlockLayout bl = block_layout(count);
  cudaStream_t s = (cudaStream_t)stream;
  void* block = nullptr;
  cudaError_t e = cudaMallocAsync(&block, bl.total, s);
  if (e != cudaSuccess) return set_cuda_error(e);
  char* blk = static_cast<char*>(block);
  e = cudaMemcpyAsync(blk + bl.jobs, jobs.data(), count * sizeof(JobDesc), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(blk + bl.order, order.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(blk + bl.ctr, 0, bl.total - bl.ctr, s);
  if (e == cudaSuccess) rc = launch_runs(blk, bl, runs, mixed, nullptr, s, &e);
  cudaError_t e2 = cudaFreeAsync(block, s);
  if (rc) return rc;
  if (e != cudaSuccess) return set_cuda_error(e);
  if (e2 != cudaSuccess) return set_cuda_error(e2);
  return MALBEC_OK;
}

int malbec_plan_create(const malbec_bundle* bundles, uint32_t count, malbec_precision prec, malbec_plan** plan) {
  if (!plan) return MALBEC_EINVAL;
  *plan = nullptr;
  std::vector<JobDesc> jobs;
  std::vector<uint32_t> order;
  std::vector<ClassRun> runs;
  uint64_t total = 0;
  int rc = build_jobs(bundles, count, prec, jobs, order, runs, &total);
  if (rc) return rc;
  malbec_plan* P = new malbec_plan();
  cudaGetDevice(&P->device);
  P->count = count;
  P->total_rays = total;
  P->mixed = prec == MALBEC_FP32_MIXED;
  P->runs = runs;
  P->bl = block_layout(count);
  cudaError_t e = cudaMalloc(&P->block, P->bl.total);
  if (e != cudaSuccess) {
    delete P;
    return set_cuda_error(e);
  }
  char* blk = static_cast<char*>(P->block);
  e = cudaMemcpy(blk + P->bl.jobs, jobs.data(), count * sizeof(JobDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(blk + P->bl.order, order.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(P->block);
    delete P;
    return set_cuda_error(e);
  }
  malbec_launch_config cfg;
  malbec_get_launch_config(&cfg);
  rc = record_plan(P, cfg);
  if (rc) {
    malbec_plan_destroy(P);
    return rc;
  }
  *plan = P;
  return MALBEC_OK;
}

int malbec_plan_launch(malbec_plan* plan, malbec_stream stream) {
  if (!plan || !plan->exec) return MALBEC_EINVAL;
  cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int malbec_plan_autotune(malbec_plan* plan, malbec_stream stream, malbec_launch_config* best) {
  if (!plan) return MALBEC_EINVAL;
  // Candidates: block size x blocks per SM (4 or 8 resident warps per SM for
  // FP64; 8 or 12 for the FP32 path), refill granularity (dead lanes a warp
  // waits for before it claims new rays: 1, 4, or 32 for whole-warp refills)
  // and, for FP32_MIXED, the FP64-zone batch and the block ray exchange on or
  // off.
  std::vector<malbec_launch_config> cand;
  if (!plan->mixed) {
    for (uint32_t rm : {1u, 4u}) cand.push_back({128u, 1u, rm, 0u, 0u, 0u});
    cand.push_back({64u, 2u, 1u, 0u, 0u, 0u});
    cand.push_back({128u, 2u, 1u, 0u, 0u, 0u});
    cand.push_back({256u, 1u, 1u, 0u, 0u, 0u});
    cand.push_back({32u, 4u, 1u, 0u, 0u, 0u});
  } else {
    const uint32_t shapes[3][2] = {{128u, 2u}, {256u, 1u}, {128u, 3u}};
    for (const auto& sh : shapes)
      for (uint32_t z = 0; z < 2; ++z)
        for (uint32_t x = 1; x <= 2; ++x) cand.push_back({sh[0], sh[1], 1u, z ? 16u : 8u, z ? 256u : 64u, x});
    cand.push_back({128u, 2u, 4u, 8u, 64u, 1u});
    // whole-warp refills: 32 neighbouring rays of a job start together
    cand.push_back({128u, 2u, 32u, 8u, 64u, 2u});
    cand.push_back({128u, 2u, 32u, 16u, 256u, 1u});
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // one replay of candidate c after `warm` untimed ones: its time in ms
  auto time_candidate = [&](const malbec_launch_config& c, int warm, float* ms) -> int {
    int r = record_plan(plan, c);
    if (r) return r;
    cudaError_t e = cudaSuccess;
    for (int w = 0; w < warm && e == cudaSuccess; ++w) e = cudaGraphLaunch(plan->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = cudaGraphLaunch(plan->exec, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaEventElapsedTime(ms, e0, e1);
    return MALBEC_OK;
  };
  // every candidate once (after a warm-up replay), then the three fastest
  // twice more: a candidate's time is the best of its replays, so a single
  // disturbed replay does not decide the choice
  std::vector<float> best_of(cand.size(), 1e30f);
  int rc = MALBEC_OK;
  for (size_t i = 0; i < cand.size() && rc == MALBEC_OK; ++i) rc = time_candidate(cand[i], 1, &best_of[i]);
  std::vector<size_t> order(cand.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return best_of[x] < best_of[y]; });
  for (size_t k = 0; k < order.size() && k < 3 && rc == MALBEC_OK; ++k)
    for (int rep = 0; rep < 2 && rc == MALBEC_OK; ++rep) {
      float ms = 0.f;
      rc = time_candidate(cand[order[k]], 0, &ms);
      if (rc == MALBEC_OK && ms < best_of[order[k]]) best_of[order[k]] = ms;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  size_t bi = 0;
  for (size_t i = 1; i < cand.size(); ++i)
    if (best_of[i] < best_of[bi]) bi = i;
  const malbec_launch_config best_cfg = cand.empty() ? plan->cfg : cand[bi];
  rc = record_plan(plan, best_cfg);
  if (rc == MALBEC_OK && best) *best = best_cfg;
  return rc;
}

int malbec_plan_destroy(malbec_plan* plan) {
  if (!plan) return MALBEC_EINVAL;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->block) cudaFree(plan->block);
  delete plan;
  return MALBEC_OK;
}

}  // extern "C"

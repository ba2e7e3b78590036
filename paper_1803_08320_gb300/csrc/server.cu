// server.cu -- the request loop: continuous batching of bundle jobs on one
// resident trace kernel (host side; the device side is the kSrcServe mode of
// trace_kernel).
//
// Host <-> device protocol:
//  - job descriptors live in a device ring of kRing slots (slot = id % kRing);
//    the host writes a slot (descriptor + zeroed counters) on its control
//    stream and waits for that copy before publishing the id;
//  - the active list (ids, smallest estimated job first), its length and the
//    stop flag live in device memory: the host builds them in pinned memory
//    and copies them on its control stream, so the kernel's look at the list
//    never leaves the GPU; it reads them with volatile loads and validates
//    every id against the slot's descriptor, so a list being rewritten can at
//    worst hide a job for one look;
//  - the last ray of a job writes the job id into done_flags[slot] (mapped
//    host memory) after a system-scope fence;
//  - the stop flag ends claiming; the kernel also leaves by itself when all
//    its warps have been idle for idle_timeout_s (each idle warp parks in a
//    device word; the warp that sees every warp parked closes the kernel and
//    all leave, so a job is never left to a partly exited grid).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <deque>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace malbec {
namespace {

constexpr uint32_t kRing = 65536;

enum JobState { kPending = 0, kActive = 1, kDone = 2 };

struct Job {
  uint64_t id = 0;
  malbec_bundle spec;
  size_t bytes = 0;
  void* out = nullptr;
  double cost = 0.0;
  int state = kPending;
};

}  // namespace
}  // namespace malbec

using namespace malbec;

struct malbec_server {
  std::mutex mu;
  malbec_server_config cfg;
  int device = 0;
  cudaStream_t compute = nullptr, control = nullptr;
  cudaEvent_t kernel_done = nullptr;
  bool launched = false;
  cudaMemPool_t pool = nullptr;
  JobDesc* d_ring = nullptr;
  JobCounter* d_ctr = nullptr;
  // active list: [count, stop] then the ids; built in pinned host memory,
  // copied to the device
  uint64_t* h_list = nullptr;
  uint64_t* d_list = nullptr;
  uint32_t stop = 0;
  // done flags, one per ring slot, in mapped host memory
  uint64_t* h_done = nullptr;
  uint64_t* d_done = nullptr;  // device alias of h_done
  unsigned long long* d_park = nullptr;  // park word of the running kernel
  uint64_t next_id = 1;
  std::unordered_map<uint64_t, Job> jobs;
  std::deque<uint64_t> pending;
  std::vector<uint64_t> active;
  size_t in_use = 0;
  malbec_server_stats stats;
};

namespace {

// Republish the active list, smallest estimated job first, with the stop
// flag: build it in pinned memory, copy it to the device and wait for the
// copy (the pinned buffer is reused by the next publish).
int publish_active(malbec_server* S) {
  std::stable_sort(S->active.begin(), S->active.end(),
                   [&](uint64_t x, uint64_t y) { return S->jobs[x].cost < S->jobs[y].cost; });
  const uint32_t k = (uint32_t)S->active.size();
  uint32_t* hdr = reinterpret_cast<uint32_t*>(S->h_list);
  hdr[0] = k;
  hdr[1] = S->stop;
  for (uint32_t i = 0; i < k; ++i) S->h_list[1 + i] = S->active[i];
  cudaError_t e = cudaMemcpyAsync(S->d_list, S->h_list, (size_t)(k + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice,
                                  S->control);
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->control);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int launch_kernel(malbec_server* S) {
  TraceParams p;
  memset(&p, 0, sizeof(p));
  p.M = 1.0;
  p.stride = 1;
  p.n = 1ull << 40;
  p.jobs = S->d_ring;
  p.job_ctr = S->d_ctr;
  p.n_jobs = kRing;
  p.active_ids = reinterpret_cast<const volatile uint64_t*>(S->d_list + 1);
  p.active_count = reinterpret_cast<const volatile uint32_t*>(S->d_list);
  p.stop_flag = reinterpret_cast<const volatile uint32_t*>(S->d_list) + 1;
  p.done_flags = reinterpret_cast<volatile uint64_t*>(S->d_done);
  p.park = S->d_park;
  p.max_active = S->cfg.max_active;
  p.idle_ns = (uint64_t)(S->cfg.idle_timeout_s * 1e9);
  p.form = S->cfg.form;
  p.method = S->cfg.method;
  fill_zone(p);
  const bool mixed = S->cfg.precision == MALBEC_FP32_MIXED;
  LaunchShape shape;
  int refill_min = 1;
  int rc = choose_shape(true, mixed, kSrcServe, kSinkJobs, p.n, &shape, &refill_min);
  if (rc) return rc;
  p.refill_min = 1;
  cudaError_t e = cudaMemsetAsync(S->d_park, 0, sizeof(unsigned long long), S->compute);
  if (e == cudaSuccess) e = launch_trace(p, true, mixed, kSrcServe, kSinkJobs, shape, S->compute);
  if (e == cudaSuccess) e = cudaEventRecord(S->kernel_done, S->compute);
  if (e != cudaSuccess) return set_cuda_error(e);
  S->launched = true;
  S->stats.kernel_launches++;
  return MALBEC_OK;
}

// (Re)launch the kernel when there is work and no instance is running.
int ensure_kernel(malbec_server* S) {
  if (S->active.empty()) return MALBEC_OK;
  if (S->launched) {
    const cudaError_t q = cudaEventQuery(S->kernel_done);
    if (q == cudaErrorNotReady) return MALBEC_OK;
    if (q != cudaSuccess) return set_cuda_error(q);
  }
  return launch_kernel(S);
}

// Admit pending jobs while the active set and the budget allow.
int admit(malbec_server* S) {
  bool changed = false;
  while (!S->pending.empty() && S->active.size() < S->cfg.max_active) {
    Job& J = S->jobs[S->pending.front()];
    if (S->in_use + J.bytes > S->cfg.hbm_budget) break;
    // the ring slot is still held by the job kRing ids older (not released yet)
    if (J.id > kRing && S->jobs.count(J.id - kRing)) break;
    cudaError_t e = cudaMallocFromPoolAsync(&J.out, J.bytes, S->pool, S->control);
    if (e != cudaSuccess) return set_cuda_error(e);
    JobDesc desc;
    fill_job_desc(J.spec, S->cfg.precision, J.out, J.id, &desc, &J.cost);
    const uint32_t slot = (uint32_t)(J.id % kRing);
    e = cudaMemcpyAsync(S->d_ring + slot, &desc, sizeof(JobDesc), cudaMemcpyHostToDevice, S->control);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->d_ctr + slot, 0, sizeof(JobCounter), S->control);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->control);
    if (e != cudaSuccess) return set_cuda_error(e);
    S->in_use += J.bytes;
    J.state = kActive;
    S->active.push_back(J.id);
    S->pending.pop_front();
    S->stats.admitted++;
    changed = true;
  }
  if (changed) return publish_active(S);
  return MALBEC_OK;
}

// Move jobs whose completion flag is set from the active list to done.
int reap(malbec_server* S) {
  bool changed = false;
  for (size_t i = 0; i < S->active.size();) {
    const uint64_t id = S->active[i];
    const volatile uint64_t* f = S->h_done + (id % kRing);
    if (*f == id) {
      S->jobs[id].state = kDone;
      S->stats.completed++;
      S->active.erase(S->active.begin() + i);
      changed = true;
    } else {
      ++i;
    }
  }
  if (changed) return publish_active(S);
  return MALBEC_OK;
}

}  // namespace

extern "C" {

int malbec_server_create(const malbec_server_config* cfg, malbec_server** server) {
  if (!cfg || !server) return MALBEC_EINVAL;
  *server = nullptr;
  if (cfg->max_active == 0 || cfg->max_active > 4096 || cfg->max_pending == 0 || cfg->hbm_budget == 0 ||
      !(cfg->idle_timeout_s > 0.0) || !isfinite(cfg->idle_timeout_s) ||
      (cfg->precision != MALBEC_FP64 && cfg->precision != MALBEC_FP32_MIXED))
    return MALBEC_EINVAL;
  // the class of jobs this server runs: any form, either method (each job's
  // tolerances are checked when it is submitted)
  if (cfg->form > MALBEC_FORM_ADM || cfg->method > MALBEC_METHOD_DOPRI5) return MALBEC_EINVAL;
  malbec_server* S = new malbec_server();
  S->cfg = *cfg;
  memset(&S->stats, 0, sizeof(S->stats));
  cudaError_t e = cudaGetDevice(&S->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->control, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->kernel_done, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    e = cudaMemPoolCreate(&S->pool, &props);
    if (e == cudaSuccess) {
      uint64_t thr = cfg->hbm_budget;
      cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&S->d_ring, (size_t)kRing * sizeof(JobDesc));
  if (e == cudaSuccess) e = cudaMalloc(&S->d_ctr, (size_t)kRing * sizeof(JobCounter));
  if (e == cudaSuccess) e = cudaMemset(S->d_ring, 0, (size_t)kRing * sizeof(JobDesc));
  if (e == cudaSuccess) e = cudaMemset(S->d_ctr, 0, (size_t)kRing * sizeof(JobCounter));
  const size_t list_bytes = (size_t)(cfg->max_active + 1) * sizeof(uint64_t);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_list, list_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&S->d_park, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(S->d_list, 0, list_bytes);
  if (e == cudaSuccess) e = cudaHostAlloc(&S->h_list, list_bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&S->h_done, (size_t)kRing * sizeof(uint64_t), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&S->d_done, S->h_done, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    int rc = set_cuda_error(e);
    malbec_server_destroy(S);
    return rc;
  }
  memset(S->h_list, 0, list_bytes);
  memset(S->h_done, 0, (size_t)kRing * sizeof(uint64_t));
  *server = S;
  return MALBEC_OK;
}

int malbec_server_destroy(malbec_server* S) {
  if (!S) return MALBEC_EINVAL;
  if (S->h_list && S->d_list && S->control) {
    // stop claiming: copy the list header with the stop flag set
    S->stop = 1u;
    uint32_t* hdr = reinterpret_cast<uint32_t*>(S->h_list);
    hdr[1] = 1u;
    if (cudaMemcpyAsync(S->d_list, S->h_list, sizeof(uint64_t), cudaMemcpyHostToDevice, S->control) == cudaSuccess)
      cudaStreamSynchronize(S->control);
  }
  if (S->compute) cudaStreamSynchronize(S->compute);
  if (S->control) cudaStreamSynchronize(S->control);
  for (auto& kv : S->jobs)
    if (kv.second.out) cudaFreeAsync(kv.second.out, S->control);
  if (S->control) cudaStreamSynchronize(S->control);
  if (S->pool) cudaMemPoolDestroy(S->pool);
  if (S->d_ring) cudaFree(S->d_ring);
  if (S->d_ctr) cudaFree(S->d_ctr);
  if (S->d_list) cudaFree(S->d_list);
  if (S->d_park) cudaFree(S->d_park);
  if (S->h_list) cudaFreeHost(S->h_list);
  if (S->h_done) cudaFreeHost(S->h_done);
  if (S->kernel_done) cudaEventDestroy(S->kernel_done);
  if (S->compute) cudaStreamDestroy(S->compute);
  if (S->control) cudaStreamDestroy(S->control);
  delete S;
  return MALBEC_OK;
}

int malbec_submit(malbec_server* S, const malbec_bundle* job, uint64_t* job_id) {
  if (!S || !job || !job_id) return MALBEC_EINVAL;
  // a job of another class than the server's (form, method) is refused
  if (job->term.form != S->cfg.form || job->term.method != S->cfg.method) return MALBEC_EINVAL;
  int rc = validate_job(*job, S->cfg.precision);
  if (rc) return rc;
  const size_t bytes = malbec_bundle_out_bytes(job, S->cfg.precision);
  if (bytes == 0 || bytes > S->cfg.hbm_budget) return MALBEC_ENOMEM;
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->pending.size() >= S->cfg.max_pending) return MALBEC_EBUSY;
  Job J;
  J.id = S->next_id++;
  J.spec = *job;
  J.spec.out = nullptr;
  J.bytes = bytes;
  S->jobs[J.id] = J;
  S->pending.push_back(J.id);
  S->stats.submitted++;
  *job_id = J.id;
  rc = admit(S);
  if (rc) return rc;
  return ensure_kernel(S);
}

int malbec_poll(malbec_server* S, uint64_t job_id, int* done) {
  if (!S || !done) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MALBEC_ENOTFOUND;
  int rc = reap(S);
  if (rc) return rc;
  rc = admit(S);
  if (rc) return rc;
  rc = ensure_kernel(S);
  if (rc) return rc;
  *done = it->second.state == kDone;
  return MALBEC_OK;
}

int malbec_job_output(malbec_server* S, uint64_t job_id, void** out, size_t* bytes) {
  if (!S || !out || !bytes) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MALBEC_ENOTFOUND;
  if (it->second.state != kDone) return MALBEC_EBUSY;
  *out = it->second.out;
  *bytes = it->second.bytes;
  return MALBEC_OK;
}

int malbec_job_copy_output(malbec_server* S, uint64_t job_id, void* dst, size_t bytes, malbec_stream stream) {
  if (!S || !dst) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MALBEC_ENOTFOUND;
  if (it->second.state != kDone) return MALBEC_EBUSY;
  if (bytes != it->second.bytes) return MALBEC_EINVAL;
  cudaError_t e = cudaMemcpyAsync(dst, it->second.out, bytes, cudaMemcpyDefault, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

int malbec_job_release(malbec_server* S, uint64_t job_id) {
  if (!S) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MALBEC_ENOTFOUND;
  if (it->second.state != kDone) return MALBEC_EBUSY;
  // the caller's copies on other streams were ordered before this call by
  // the caller; free in the control stream after them
  cudaError_t e = cudaFreeAsync(it->second.out, S->control);
  if (e != cudaSuccess) return set_cuda_error(e);
  S->in_use -= it->second.bytes;
  S->jobs.erase(it);
  S->stats.released++;
  int rc = admit(S);
  if (rc) return rc;
  return ensure_kernel(S);
}

int malbec_server_stats_get(malbec_server* S, malbec_server_stats* st) {
  if (!S || !st) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->stats;
  st->pending = S->pending.size();
  st->active = S->active.size();
  st->bytes_in_use = S->in_use;
  return MALBEC_OK;
}

}  // extern "C"

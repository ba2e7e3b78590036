// noalloc.cu -- malbec_trace_noalloc: malbec_trace without any device
// allocation.
//
// malbec_trace takes its 256-byte work-queue block from the stream-ordered
// allocator on every call.  Some callers cannot allocate device memory at
// all: code running inside a CUDA graph that is being captured with a mode
// that forbids allocation calls, real-time loops that must never touch the
// allocator (an allocation can synchronise or grow a memory pool at an
// unpredictable moment), and embedders that own every byte of device memory
// through their own arena and forbid libraries from calling cudaMalloc.
// For them this entry point runs the same kernel with its work-queue block
// in a file-scope __device__ array of MALBEC_NOALLOC_SCRATCH_BYTES bytes that
// every GPU which loads the library holds until the process exits.
#include <string.h>

#include <mutex>

#include "internal.h"

namespace malbec {
namespace {

// The kernel's work-queue block lives here.  In host code this name is only
// a stand-in for the device object: its device address is looked up with
// cudaGetSymbolAddress once per CUDA context (in practice once per device,
// in the device's primary context).
__device__ __align__(256) unsigned char g_noalloc_scratch[MALBEC_NOALLOC_SCRATCH_BYTES];

// Scratch one trace launch needs: the work-queue counter block (the same
// size malbec_trace allocates), independent of the number of rays.  It fits
// the static block by construction, so this call never returns
// MALBEC_ESCRATCH; the code is kept for entry points with larger scratch.
constexpr size_t kTraceScratchBytes = 256;
static_assert(kTraceScratchBytes <= MALBEC_NOALLOC_SCRATCH_BYTES, "the work-queue block fits the static array");

std::mutex g_mu;

// The address is cached per CUDA context, keyed by the context's id
// (cuCtxGetId: unique over the life of the process), so that a context
// created after cudaDeviceReset -- which unloads this library's device code
// and with it the array -- looks the address up again instead of reusing a
// stale one.  The two driver calls are reached through the runtime
// (cudaGetDriverEntryPointByVersion), so the library does not link libcuda.
struct CtxScratch {
  unsigned long long ctx_id;
  void* ptr;
};
constexpr int kCtxSlots = 64;
CtxScratch g_slots[kCtxSlots];
int g_next_slot = 0;

typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

// The id of the calling thread's current context, creating the device's
// primary context first if there is none yet (cudaGetSymbolAddress does that
// as a side effect: no allocation call is made).
int current_ctx_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f1)
      return set_cuda_error(e != cudaSuccess ? e : cudaErrorNotSupported);
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !f2)
      return set_cuda_error(e != cudaSuccess ? e : cudaErrorNotSupported);
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  void* ctx = nullptr;
  if (get_current(&ctx) != 0) return set_cuda_error(cudaErrorDeviceUninitialized);
  if (!ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return set_cuda_error(e);
    if (get_current(&ctx) != 0 || !ctx) return set_cuda_error(cudaErrorDeviceUninitialized);
  }
  if (get_id(ctx, id) != 0) return set_cuda_error(cudaErrorDeviceUninitialized);
  return MALBEC_OK;
}

// Device address of g_noalloc_scratch in the current context, looked up on
// the first call in that context (with its device current).
int scratch_address(void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long id = 0;
  int rc = current_ctx_id(&id);
  if (rc) return rc;
  for (int k = 0; k < kCtxSlots; ++k) {
    if (g_slots[k].ptr && g_slots[k].ctx_id == id) {
      *out = g_slots[k].ptr;
      return MALBEC_OK;
    }
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return set_cuda_error(e);
  g_slots[g_next_slot] = CtxScratch{id, p};
  g_next_slot = (g_next_slot + 1) % kCtxSlots;
  *out = p;
  return MALBEC_OK;
}

}  // namespace
}  // namespace malbec

using namespace malbec;

extern "C" int malbec_trace_noalloc(malbec_metric m, const double* ics, uint64_t n, malbec_term t,
                                    malbec_out_mode mode, uint32_t stride, malbec_precision prec, void* out,
                                    malbec_stream stream) {
  int rc = check_metric(m);
  if (rc) return rc;
  rc = check_term(t, m);
  if (rc) return rc;
  rc = check_method_precision(t, prec);
  if (rc) return rc;
  if (!ics || !out) return MALBEC_EINVAL;
  malbec_layout L;
  rc = malbec_out_layout(mode, prec, n, t.n_steps_cap, stride, &L);
  if (rc) return rc;
  if (((uintptr_t)out & 255u) != 0) return MALBEC_EINVAL;
  char* o = static_cast<char*>(out);
  TraceParams p;
  memset(&p, 0, sizeof(p));
  p.M = m.M;
  p.a = m.a;
  p.a_per_ray = m.a_per_ray;
  p.eps_hor = t.eps_hor;
  p.r_esc = t.r_esc;
  p.dl = t.dl;
  p.dl_r_scale = t.dl_r_scale;
  p.form = t.form;
  p.method = t.method;
  p.rtol = t.rtol;
  p.atol = t.atol;
  p.cap = t.n_steps_cap;
  p.ics = ics;
  p.n = n;
  p.y_out = reinterpret_cast<double*>(o + L.y);
  p.lambda_out = reinterpret_cast<double*>(o + L.lambda);
  p.inv0_out = reinterpret_cast<double*>(o + L.inv0);
  p.inv1_out = reinterpret_cast<double*>(o + L.inv1);
  p.steps_out = reinterpret_cast<uint32_t*>(o + L.steps);
  p.fate_out = reinterpret_cast<uint8_t*>(o + L.fate);
  const bool strided = mode != MALBEC_OUT_FINAL;
  p.traj = strided ? static_cast<void*>(o + L.traj) : nullptr;
  p.stride = strided ? stride : 1;
  p.n_samples = L.n_samples;
  p.traj_cartesian = mode == MALBEC_OUT_STRIDED_CARTESIAN ? 1 : 0;
  const bool kerr = !(m.a == 0.0 && m.a_per_ray == nullptr);
  const bool mixed = prec == MALBEC_FP32_MIXED;
  const Sink sink = strided ? kSinkStrided : kSinkFinal;
  LaunchShape shape;
  int refill_min = 1;
  rc = choose_shape(kerr, mixed, kSrcStates, sink, n, &shape, &refill_min);
  if (rc) return rc;
  p.refill_min = refill_min;
  fill_zone(p);
  void* scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc) return rc;
  // the block keeps the previous call's counter: the queue head must start at zero
  cudaError_t e = cudaMemsetAsync(scratch, 0, kTraceScratchBytes, (cudaStream_t)stream);
  if (e != cudaSuccess) return set_cuda_error(e);
  p.head = static_cast<unsigned long long*>(scratch);
  e = launch_trace(p, kerr, mixed, kSrcStates, sink, shape, (cudaStream_t)stream);
  return e == cudaSuccess ? MALBEC_OK : set_cuda_error(e);
}

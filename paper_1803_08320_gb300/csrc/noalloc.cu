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
// a stand-in for the device object: its device address is looked up once
// per device with cudaGetSymbolAddress.
__device__ __align__(256) unsigned char g_noalloc_scratch[MALBEC_NOALLOC_SCRATCH_BYTES];

// Scratch one trace launch needs: the work-queue counter block (the same
// size malbec_trace allocates), independent of the number of rays.
constexpr size_t kTraceScratchBytes = 256;

std::mutex g_mu;
void* g_scratch_ptr[64];

// Device address of g_noalloc_scratch on the current device, looked up on
// the first call for that device (with that device current).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  if (dev < 0 || dev >= 64) return MALBEC_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return set_cuda_error(e);
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
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
  if (kTraceScratchBytes > MALBEC_NOALLOC_SCRATCH_BYTES) return MALBEC_ESCRATCH;
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
  p.traj = mode == MALBEC_OUT_STRIDED ? static_cast<void*>(o + L.traj) : nullptr;
  p.stride = mode == MALBEC_OUT_STRIDED ? stride : 1;
  p.n_samples = L.n_samples;
  const bool kerr = !(m.a == 0.0 && m.a_per_ray == nullptr);
  const bool mixed = prec == MALBEC_FP32_MIXED;
  const Sink sink = mode == MALBEC_OUT_STRIDED ? kSinkStrided : kSinkFinal;
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

// trace.cu -- the RK4 instantiations of the trace kernel (trace_kernel.cuh),
// the kernel dispatch and the launch.
#include "trace_kernel.cuh"

namespace malbec {
namespace {

const void* pick(bool kerr, bool mixed, Source src, Sink sink, bool banks, int form, int method) {
  // Dormand-Prince 5(4): the kernels of trace_dopri.cu
  if (method == MALBEC_METHOD_DOPRI5) return pick_dopri(mixed, src, sink, form);
  // canonical forms (Sec. 2, eq. Ham, with g of eq. kerr or of eq. ADM):
  // every source
  if (form != MALBEC_FORM_GEODESIC) {
#define MALBEC_PICK_HAM(F, S, T)                                                                   \
  if (form == F && src == S && sink == T) {                                                        \
    if (!mixed) return kernel_ptr<true, false, S, T, false, F>();                                  \
    return banks ? kernel_ptr<true, true, S, T, true, F>() : kernel_ptr<true, true, S, T, false, F>(); \
  }
    MALBEC_PICK_HAM(MALBEC_FORM_HAMILTONIAN, kSrcStates, kSinkFinal)
    MALBEC_PICK_HAM(MALBEC_FORM_HAMILTONIAN, kSrcStates, kSinkStrided)
    MALBEC_PICK_HAM(MALBEC_FORM_HAMILTONIAN, kSrcCamera, kSinkCamera)
    MALBEC_PICK_HAM(MALBEC_FORM_ADM, kSrcStates, kSinkFinal)
    MALBEC_PICK_HAM(MALBEC_FORM_ADM, kSrcStates, kSinkStrided)
    MALBEC_PICK_HAM(MALBEC_FORM_ADM, kSrcCamera, kSinkCamera)
    MALBEC_PICK_HAM(MALBEC_FORM_HAMILTONIAN, kSrcJobs, kSinkJobs)
    MALBEC_PICK_HAM(MALBEC_FORM_ADM, kSrcJobs, kSinkJobs)
    MALBEC_PICK_HAM(MALBEC_FORM_HAMILTONIAN, kSrcServe, kSinkJobs)
    MALBEC_PICK_HAM(MALBEC_FORM_ADM, kSrcServe, kSinkJobs)
#undef MALBEC_PICK_HAM
    return nullptr;
  }
#define MALBEC_PICK(K, X, S, T)                                                        \
  if (kerr == K && mixed == X && src == S && sink == T) {                              \
    if (X && banks) return kernel_ptr<K, X, S, T, X>();                               \
    return kernel_ptr<K, X, S, T, false>();                                            \
  }
  MALBEC_PICK(true, false, kSrcJobs, kSinkJobs)
  MALBEC_PICK(true, true, kSrcJobs, kSinkJobs)
  MALBEC_PICK(true, false, kSrcServe, kSinkJobs)
  MALBEC_PICK(true, true, kSrcServe, kSinkJobs)
  MALBEC_PICK(false, false, kSrcStates, kSinkFinal)
  MALBEC_PICK(true, false, kSrcStates, kSinkFinal)
  MALBEC_PICK(false, true, kSrcStates, kSinkFinal)
  MALBEC_PICK(true, true, kSrcStates, kSinkFinal)
  MALBEC_PICK(false, false, kSrcStates, kSinkStrided)
  MALBEC_PICK(true, false, kSrcStates, kSinkStrided)
  MALBEC_PICK(false, true, kSrcStates, kSinkStrided)
  MALBEC_PICK(true, true, kSrcStates, kSinkStrided)
  MALBEC_PICK(false, false, kSrcCamera, kSinkCamera)
  MALBEC_PICK(true, false, kSrcCamera, kSinkCamera)
  MALBEC_PICK(false, true, kSrcCamera, kSinkCamera)
  MALBEC_PICK(true, true, kSrcCamera, kSinkCamera)
#undef MALBEC_PICK
  return nullptr;
}

}  // namespace

cudaError_t read_wait_timeouts(unsigned long long* total) {
  return cudaMemcpyFromSymbol(total, g_wait_timeouts, sizeof(unsigned long long));
}

int trace_max_blocks_per_sm(bool kerr, bool mixed, Source src, Sink sink, bool banks, int threads_per_block,
                            int form, int method) {
  const void* k = pick(kerr, mixed, src, sink, mixed && banks && method == MALBEC_METHOD_RK4, form, method);
  if (!k) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads_per_block, 0) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_trace(const TraceParams& p, bool kerr, bool mixed, Source src, Sink sink,
                         const LaunchShape& shape, cudaStream_t stream) {
  // automatic block exchange: on for job tables, the request loop and state
  // arrays (mixes of long timelike orbits spend many steps in the polar FP64
  // zone), off for whole-image cameras (too few steps in their zone to pay
  // for a zone warp)
  const int exchange = p.method == MALBEC_METHOD_DOPRI5 ? 0 : (p.exchange >= 0 ? p.exchange : (src == kSrcCamera ? 0 : 1));
  const void* k = pick(kerr, mixed, src, sink, mixed && exchange == 1, (int)p.form, (int)p.method);
  if (!k) return cudaErrorInvalidValue;
  // automatic FP64-zone batch: 8 lanes with the exchange (a warp hands fewer
  // zone rays to the zone warp), a full warp without it (a zone step then
  // waits for 32 lanes, zone_wait warp steps, or a warp with no FP32 lane)
  TraceParams q = p;
  if (q.zone_batch < 0) q.zone_batch = exchange == 1 ? 8 : 32;
  if (shape.threads_per_block <= 0 || shape.threads_per_block > kMaxTPB ||
      shape.threads_per_block % 32 != 0 || shape.blocks <= 0)
    return cudaErrorInvalidConfiguration;
  void* args[] = {&q};
  return cudaLaunchKernel(k, dim3(shape.blocks), dim3(shape.threads_per_block), args, 0, stream);
}

}  // namespace malbec

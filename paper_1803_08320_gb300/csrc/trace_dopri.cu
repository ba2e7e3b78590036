// trace_dopri.cu -- the Dormand-Prince 5(4) instantiations of the trace
// kernel (trace_kernel.cuh), in a translation unit of their own so that the
// library's kernels compile in parallel.
#include "trace_kernel.cuh"

namespace malbec {

const void* pick_dopri(bool mixed, Source src, Sink sink, int form) {
  // Dormand-Prince 5(4): every form (the Kerr right-hand sides, a = 0
  // included), every source, FP64 and FP32_MIXED (no block exchange: a ray
  // never changes warps, so its step-size state stays in its lane)
  if (mixed) {
#define MALBEC_PICK_DPM(F)                                                                 \
  if (form == F) {                                                                         \
    if (src == kSrcStates && sink == kSinkFinal)                                           \
      return kernel_ptr<true, true, kSrcStates, kSinkFinal, false, F, MALBEC_METHOD_DOPRI5>();    \
    if (src == kSrcStates && sink == kSinkStrided)                                         \
      return kernel_ptr<true, true, kSrcStates, kSinkStrided, false, F, MALBEC_METHOD_DOPRI5>();  \
    if (src == kSrcCamera && sink == kSinkCamera)                                          \
      return kernel_ptr<true, true, kSrcCamera, kSinkCamera, false, F, MALBEC_METHOD_DOPRI5>();   \
    if (src == kSrcJobs && sink == kSinkJobs)                                              \
      return kernel_ptr<true, true, kSrcJobs, kSinkJobs, false, F, MALBEC_METHOD_DOPRI5>();       \
    if (src == kSrcServe && sink == kSinkJobs)                                             \
      return kernel_ptr<true, true, kSrcServe, kSinkJobs, false, F, MALBEC_METHOD_DOPRI5>();      \
  }
    MALBEC_PICK_DPM(MALBEC_FORM_GEODESIC)
    MALBEC_PICK_DPM(MALBEC_FORM_HAMILTONIAN)
    MALBEC_PICK_DPM(MALBEC_FORM_ADM)
#undef MALBEC_PICK_DPM
    return nullptr;
  }
#define MALBEC_PICK_DP(F)                                                                  \
  if (form == F) {                                                                         \
    if (src == kSrcStates && sink == kSinkFinal)                                           \
      return kernel_ptr<true, false, kSrcStates, kSinkFinal, false, F, MALBEC_METHOD_DOPRI5>();   \
    if (src == kSrcStates && sink == kSinkStrided)                                         \
      return kernel_ptr<true, false, kSrcStates, kSinkStrided, false, F, MALBEC_METHOD_DOPRI5>(); \
    if (src == kSrcCamera && sink == kSinkCamera)                                          \
      return kernel_ptr<true, false, kSrcCamera, kSinkCamera, false, F, MALBEC_METHOD_DOPRI5>();  \
    if (src == kSrcJobs && sink == kSinkJobs)                                              \
      return kernel_ptr<true, false, kSrcJobs, kSinkJobs, false, F, MALBEC_METHOD_DOPRI5>();      \
    if (src == kSrcServe && sink == kSinkJobs)                                             \
      return kernel_ptr<true, false, kSrcServe, kSinkJobs, false, F, MALBEC_METHOD_DOPRI5>();     \
  }
  MALBEC_PICK_DP(MALBEC_FORM_GEODESIC)
  MALBEC_PICK_DP(MALBEC_FORM_HAMILTONIAN)
  MALBEC_PICK_DP(MALBEC_FORM_ADM)
#undef MALBEC_PICK_DP
  return nullptr;
}

}  // namespace malbec

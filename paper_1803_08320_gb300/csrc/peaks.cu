// peaks.cu -- measured non-tensor FMA throughput (the roofline denominator of
// the ALU-bound geodesic kernels).  Eight independent FMA chains per thread,
// every SM busy, timed with CUDA events; best of three launches.
#include "internal.h"

namespace malbec {
namespace {

template <typename T>
__global__ void fma_peak_kernel(T* out, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(int iters, double* gflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  const int threads = 256, blocks = sms * 8;
  T* buf = nullptr;
  e = cudaMalloc(&buf, sizeof(T) * (size_t)threads * blocks);
  if (e != cudaSuccess) return set_cuda_error(e);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_peak_kernel<T><<<blocks, threads>>>(buf, 16, T(1.0000001), T(1e-9));
  float best = 1e30f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0);
    fma_peak_kernel<T><<<blocks, threads>>>(buf, iters, T(1.0000001), T(1e-9));
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return set_cuda_error(e);
  *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e6);
  return MALBEC_OK;
}

}  // namespace
}  // namespace malbec

extern "C" int malbec_measure_fma_peak(malbec_precision prec, double* gflops) {
  if (!gflops) return MALBEC_EINVAL;
  if (prec == MALBEC_FP64) return malbec::measure<double>(4000, gflops);
  if (prec == MALBEC_FP32_MIXED) return malbec::measure<float>(200000, gflops);
  return MALBEC_EINVAL;
}

// peaks.cu -- measured non-tensor FMA throughput (the roofline denominator of
// the ALU-bound geodesic kernels).  Eight independent FMA chains per thread,
// every SM busy, timed with CUDA events; best of three launches.  Also the
// bare FP64 RK4 step loop (the ceiling the trace kernels approach for their
// instruction mix) and a self-check of the FP64 stage trigonometry and
// reciprocal against CUDA's sincos and division.
#include <string.h>

#include "fp32pair.cuh"
#include "geodesic.cuh"
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

// The RK4 step of one form, nothing else: each thread follows an inclined
// bound orbit of Kerr a = 0.9 M (r0 = 10 M + a lane offset, dtau = 0.5) for
// nsteps steps; two warps per SM sub-partition, as in the FP64 trace kernels.
template <int kForm>
__global__ void __launch_bounds__(128, 2) step_loop_kernel(double* out, int nsteps, unsigned long long lane_zero) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const double M = 1.0, a = 0.9, h = 0.5;
  const BH<double> bh = make_bh<double>(M, a, (unsigned long long)threadIdx.x & lane_zero);  // as the trace kernels
  const double r0 = 10.0 + 1e-3 * (tid % 97);
  double y[8] = {0.0, r0, 1.2, 0.0, 1.0 / sqrt(1.0 - 3.0 / r0), 0.0, 0.01, 0.0};
  y[7] = sqrt(1.0 / (r0 * r0 * r0)) * y[4];
  if constexpr (kForm != MALBEC_FORM_GEODESIC) {
    double p[4];
    lower_velocity(M, a, y, p);
#pragma unroll
    for (int c = 0; c < 4; ++c) y[4 + c] = p[c];
  }
  for (int n = 0; n < nsteps; ++n) {
    if constexpr (kForm == MALBEC_FORM_GEODESIC)
      rk4_step<true, double>(bh, h, y);
    else
      rk4_step_ham<double, false, kForm>(bh, h, y);
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) acc += y[c];
  out[tid] = acc;
}

template <int kForm>
int step_loop(double* steps_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_cuda_error(e);
  const int threads = 128, blocks = 2 * sms, nsteps = 4000;  // two warps per SM sub-partition, as the trace kernels
  double* buf = nullptr;
  e = cudaMalloc(&buf, sizeof(double) * (size_t)threads * blocks);
  if (e != cudaSuccess) return set_cuda_error(e);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  step_loop_kernel<kForm><<<blocks, threads>>>(buf, 50, 0ull);
  float best = 1e30f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0);
    step_loop_kernel<kForm><<<blocks, threads>>>(buf, nsteps, 0ull);
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
  *steps_per_s = (double)nsteps * blocks * threads / (best * 1e-3);
  return MALBEC_OK;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// stage_trig against sincos at exactly representable angles th0 + d
// (th0 = k / 256 with |th0| < 4, d = m / 2^40 with |d| <= 1/4, so the sum has
// at most 42 significant bits; one eighth of the draws fall in the short
// tier |d| < 2^-5), and recip against the IEEE division on
// x = mantissa x 2^e, e in [-60, 60].  err: max |sin error|, max |cos error|,
// max recip error in units of the last place of 1/x, max relative error of
// the hardware estimate alone, and the steps' sine and cosine (Trig<double>)
// against sincos: x uniform in [-4, 8] or, every other draw, a multiple of
// pi/2 there plus an offset down to 2^-60, or (one draw in 16) up to 2^30 in
// magnitude; non-negative doubles ordered as integers.
__global__ void helpers_check_kernel(unsigned long long* err, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long h1 = mix64(2 * i), h2 = mix64(2 * i + 1);
    const double th0 = (double)((long long)(h1 % 2047ull) - 1023) / 256.0;
    const double d = (double)((long long)(h2 % ((1ull << 39) + 1ull)) - (1ll << 38)) / 1099511627776.0;
    const double th = th0 + d;
    double s0, c0, s, c, sr, cr;
    sincos(th0, &s0, &c0);
    stage_trig<double>(make_bh<double>(1.0, 0.0), s0, c0, 1.0, d, th0, &s, &c);
    sincos(th, &sr, &cr);
    const double es = fabs(s - sr), ec = fabs(c - cr);
    const unsigned long long h3 = mix64(~i);
    const double x = ldexp(1.0 + (double)(h3 >> 11) * 0x1.0p-53, (int)((h3 & 0xFFFFull) % 121ull) - 60);
    const double q = 1.0 / x, y = recip<double>(x);
    double y0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
    const double ulp = ldexp(1.0, ilogb(q) - 52);
    const double er = fabs(y - q) / ulp, e0 = fabs(y0 - q) / q;
    atomicMax(&err[0], (unsigned long long)__double_as_longlong(es));
    atomicMax(&err[1], (unsigned long long)__double_as_longlong(ec));
    atomicMax(&err[2], (unsigned long long)__double_as_longlong(er));
    atomicMax(&err[3], (unsigned long long)__double_as_longlong(e0));
    const unsigned long long h4 = mix64(i ^ 0x5bd1e995ull);
    const double u = (double)(h4 >> 11) * 0x1.0p-53;
    double xa = (h4 & 1ull) ? fma(12.0, u, -4.0)
                            : fma(1.5707963267948966, (double)((long long)((h4 >> 1) % 8ull) - 2),
                                  ldexp(u - 0.5, -(int)((h4 >> 4) % 61ull)));
    if (((h4 >> 10) & 15ull) == 0ull) xa = ldexp(u - 0.5, (int)((h4 >> 14) % 31ull));
    double sa, ca, sl, cl;
    Trig<double>::sc(make_bh<double>(1.0, 0.0), xa, &sa, &ca);
    sincos(xa, &sl, &cl);
    atomicMax(&err[4], (unsigned long long)__double_as_longlong(fabs(sa - sl)));
    atomicMax(&err[5], (unsigned long long)__double_as_longlong(fabs(ca - cl)));
  }
}


// Operand forms against the plain operations, bit for bit: FP64 fma(x, y, -0)
// against x*y, fma(x, 1, y) against x + y and fma(x, 1, -y) against x - y
// (-0 and 1 in per-thread registers, as the trace kernels hold them), twice(x)
// against x + x for finite normal x; the paired FP32 add, subtract, multiply
// and fma and comp_add2 against their scalar forms.  Operands: seeded random
// bit patterns (every class: zeros, subnormals, normals, infinities, NaN)
// and, every fourth draw, random magnitudes near each other; a NaN result
// matches a NaN result.  cnt[k]: mismatches of check k.
__device__ __forceinline__ bool same64(double a, double b) {
  return (a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same32(float a, float b) {
  return (a != a && b != b) || __float_as_int(a) == __float_as_int(b);
}
__device__ __forceinline__ double draw64(unsigned long long h, unsigned long long g) {
  if ((g & 3ull) == 0ull) return ldexp(1.0 + (double)(h >> 12) * 0x1.0p-52, (int)(h % 41ull) - 20) * ((h >> 7) & 1 ? -1.0 : 1.0);
  return __longlong_as_double((long long)h);
}
__device__ __forceinline__ float draw32(unsigned long long h, unsigned long long g) {
  if ((g & 3ull) == 0ull) return ldexpf(1.0f + (float)(h >> 41) * 0x1.0p-23f, (int)(h % 41ull) - 20) * ((h >> 7) & 1 ? -1.f : 1.f);
  return __int_as_float((int)(h >> 16));
}
__global__ void operand_forms_kernel(unsigned long long* cnt, uint64_t n, unsigned long long lane_zero) {
  const BH<double> b = make_bh<double>(1.0, 0.5, (unsigned long long)threadIdx.x & lane_zero);
  unsigned long long c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long h1 = mix64(4 * i), h2 = mix64(4 * i + 1), h3 = mix64(4 * i + 2), h4 = mix64(4 * i + 3);
    const double x = draw64(h1, h3), y = draw64(h2, h3 >> 2);
    c[0] += !same64(vmul(b, x, y), x * y);
    c[1] += !same64(vadd(b, x, y), x + y);
    c[2] += !same64(vsub(b, x, y), x - y);
    const double xn = ldexp(1.0 + (double)(h4 >> 12) * 0x1.0p-52, (int)(h4 % 2045ull) - 1022);  // finite normal
    c[3] += !same64(twice(xn), xn + xn) || !same64(twice(-xn), -xn - xn);
    const float2 p = make_float2(draw32(h1, h3), draw32(h2, h4)), q = make_float2(draw32(h3, h1), draw32(h4, h2));
    const float2 r = make_float2(draw32(h1 ^ h4, h2), draw32(h2 ^ h3, h1));
    const float2 sa = f2add(p, q), ss = f2sub(p, q), sm = f2mul(p, q), sf = f2fma(p, q, r);
    c[4] += !same32(sa.x, p.x + q.x) || !same32(sa.y, p.y + q.y);
    c[5] += !same32(ss.x, p.x - q.x) || !same32(ss.y, p.y - q.y);
    c[6] += !same32(sm.x, p.x * q.x) || !same32(sm.y, p.y * q.y) || !same32(sf.x, fmaf(p.x, q.x, r.x)) ||
            !same32(sf.y, fmaf(p.y, q.y, r.y));
    // comp_add2 on a compensated pair against comp_add per component
    float2 hi2 = make_float2(p.x, q.x), lo2 = make_float2(p.x * 0x1.0p-30f, q.x * 0x1.0p-30f);
    const float2 d2 = make_float2(r.x, r.y), e2 = make_float2(r.x * 0x1.0p-30f, r.y * 0x1.0p-30f);
    float h0 = hi2.x, l0 = lo2.x, hh = hi2.y, ll = lo2.y;
    comp_add(h0, l0, d2.x, e2.x);
    comp_add(hh, ll, d2.y, e2.y);
    comp_add2(hi2, lo2, d2, e2);
    c[7] += !same32(hi2.x, h0) || !same32(lo2.x, l0) || !same32(hi2.y, hh) || !same32(lo2.y, ll);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (c[k]) atomicAdd(&cnt[k], c[k]);
}
}  // namespace
}  // namespace malbec

extern "C" int malbec_measure_step_loop(uint32_t form, double* steps_per_s) {
  if (!steps_per_s) return MALBEC_EINVAL;
  if (form == MALBEC_FORM_GEODESIC) return malbec::step_loop<MALBEC_FORM_GEODESIC>(steps_per_s);
  if (form == MALBEC_FORM_HAMILTONIAN) return malbec::step_loop<MALBEC_FORM_HAMILTONIAN>(steps_per_s);
  if (form == MALBEC_FORM_ADM) return malbec::step_loop<MALBEC_FORM_ADM>(steps_per_s);
  return MALBEC_EINVAL;
}

extern "C" int malbec_check_fp64_helpers(double err[6]) {
  if (!err) return MALBEC_EINVAL;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 6 * sizeof(unsigned long long));
  if (e != cudaSuccess) return malbec::set_cuda_error(e);
  e = cudaMemset(d, 0, 6 * sizeof(unsigned long long));
  if (e == cudaSuccess) {
    malbec::helpers_check_kernel<<<1024, 256>>>(d, 1ull << 22);
    e = cudaGetLastError();
  }
  unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return malbec::set_cuda_error(e);
  for (int k = 0; k < 6; ++k) memcpy(&err[k], &h[k], sizeof(double));
  return MALBEC_OK;
}

extern "C" int malbec_measure_fma_peak(malbec_precision prec, double* gflops) {
  if (!gflops) return MALBEC_EINVAL;
  if (prec == MALBEC_FP64) return malbec::measure<double>(4000, gflops);
  if (prec == MALBEC_FP32_MIXED) return malbec::measure<float>(200000, gflops);
  return MALBEC_EINVAL;
}

extern "C" int malbec_check_operand_forms(uint64_t counts[8]) {
  if (!counts) return MALBEC_EINVAL;
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 8 * sizeof(unsigned long long));
  if (e != cudaSuccess) return malbec::set_cuda_error(e);
  e = cudaMemset(d, 0, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) {
    malbec::operand_forms_kernel<<<1024, 256>>>(d, 1ull << 22, 0ull);
    e = cudaGetLastError();
  }
  unsigned long long h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return malbec::set_cuda_error(e);
  for (int k = 0; k < 8; ++k) counts[k] = h[k];
  return MALBEC_OK;
}

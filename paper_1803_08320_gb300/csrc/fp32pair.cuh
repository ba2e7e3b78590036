// fp32pair.cuh -- compensated FP32 arithmetic of the FP32_MIXED state and
// the paired FP32 operations (sm_100 and later) it runs on.
#pragma once
#include <cuda_runtime.h>

namespace malbec {

// TwoSum (Knuth): s = fl(a + b) and the exact rounding error e, a + b = s + e.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += d + d_err, renormalised so that hi = fl(hi + lo): TwoSum of
// hi + d (no order of magnitudes assumed), then the error terms folded in and
// the pair renormalised with Fast2Sum, exact here because |e| (a rounding
// error of s plus the small lo and d_err) never exceeds |s| -- the same
// result as a second TwoSum in half the operations.
__device__ __forceinline__ void comp_add(float& hi, float& lo, float d, float d_err) {
  float s, e;
  two_sum(hi, d, s, e);
  e += lo + d_err;
  hi = s + e;
  lo = e - (hi - s);
}

// Paired FP32 operations (sm_100 and later: FFMA2, FADD2, FMUL2 and the PTX
// sub.rn.f32x2 act on two FP32 values per lane with one instruction, each
// rounded to nearest as the scalar operation would be).  On this part a
// paired add or multiply takes one issue for two results at the scalar
// rate of each (measured), so they halve the issue slots of vector-shaped
// FP32 work.
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 ra, rb, rr;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tsub.rn.f32x2 rr, ra, rb;\n\tmov.b64 {%0, %1}, rr;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
// comp_add on two components at once (the same operations in the same order).
__device__ __forceinline__ void comp_add2(float2& hi, float2& lo, float2 d, float2 d_err) {
  const float2 s = f2add(hi, d);
  const float2 bb = f2sub(s, hi);
  float2 e = f2add(f2sub(hi, f2sub(s, bb)), f2sub(d, bb));
  e = f2add(e, f2add(lo, d_err));
  hi = f2add(s, e);
  lo = f2sub(e, f2sub(hi, s));
}

}  // namespace malbec

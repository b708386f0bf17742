// dfloat.cuh -- double-float multiply-add for dense FP64 transforms kept
// on the FP32 pipes (the spline solve's transforms).  Internal to the
// library.
#pragma once

#include <cuda_runtime.h>

namespace pic {

// A value as an FP32 pair (hi, lo), the product by Dekker's method
// via FMA and the sum by Knuth's two-sum, ~2^-48 relative.
__device__ __forceinline__ float2 sdf_split(double x) {
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}
// (the rounded operations are spelled out so that no multiply and add are
// contracted into one FMA, which would break the error-free steps)
__device__ __forceinline__ float2 sdf_fma(float2 acc, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = __fadd_rn(acc.x, p);
  const float v = __fsub_rn(s, acc.x);
  const float t = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, v)), __fsub_rn(p, v));
  const float lo = __fadd_rn(__fadd_rn(t, e), acc.y);
  const float hi = __fadd_rn(s, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}
}  // namespace pic

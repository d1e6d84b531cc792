// Double-FP32 ("double-float") complex arithmetic: a value is an unevaluated sum
// hi + lo of two floats (about 48 significant bits).  GB300 retires 64 FP32 FMAs per
// FP64 FMA, so streaming kernels whose FP64 form is bound by the FP64 pipe run on the
// FP32 pipes in this form.  Products use the error-free transformation
// a*b = p + e with p = fl(a*b), e = fma(a, b, -p) (Dekker); sums use Knuth's
// two-sum s + t = a + b.  A complex value is a float4 (re_hi, im_hi, re_lo, im_lo).
#pragma once
#include <cuda_runtime.h>

namespace helm {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ float4 to_df(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
}

__device__ __forceinline__ double2 from_df(float4 a) {
  return make_double2((double)a.x + (double)a.z, (double)a.y + (double)a.w);
}

// acc += x * r.  acc holds the running sums: (.x, .y) high parts accumulated with two-sum,
// (.z, .w) the low parts (rounding errors of products and sums, cross terms).
__device__ __forceinline__ void df_cmac(float4& acc, float4 x, float4 r) {
  float p, e, s, t;
  // re += x.re_hi * r.re_hi
  p = x.x * r.x; e = fmaf(x.x, r.x, -p);
  two_sum(acc.x, p, s, t); acc.x = s;
  acc.z += t + e + fmaf(x.x, r.z, x.z * r.x);
  // re -= x.im_hi * r.im_hi
  p = x.y * r.y; e = fmaf(x.y, r.y, -p);
  two_sum(acc.x, -p, s, t); acc.x = s;
  acc.z += t - e - fmaf(x.y, r.w, x.w * r.y);
  // im += x.re_hi * r.im_hi
  p = x.x * r.y; e = fmaf(x.x, r.y, -p);
  two_sum(acc.y, p, s, t); acc.y = s;
  acc.w += t + e + fmaf(x.x, r.w, x.z * r.y);
  // im += x.im_hi * r.re_hi
  p = x.y * r.x; e = fmaf(x.y, r.x, -p);
  two_sum(acc.y, p, s, t); acc.y = s;
  acc.w += t + e + fmaf(x.y, r.z, x.w * r.x);
}

}  // namespace helm

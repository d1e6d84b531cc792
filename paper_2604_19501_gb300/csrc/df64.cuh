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

// acc += conj(v) * w (same accumulator convention as df_cmac)
__device__ __forceinline__ void df_cmacc(float4& acc, float4 v, float4 w) {
  float p, e, s, t;
  // re += v.re * w.re
  p = v.x * w.x; e = fmaf(v.x, w.x, -p);
  two_sum(acc.x, p, s, t); acc.x = s;
  acc.z += t + e + fmaf(v.x, w.z, v.z * w.x);
  // re += v.im * w.im
  p = v.y * w.y; e = fmaf(v.y, w.y, -p);
  two_sum(acc.x, p, s, t); acc.x = s;
  acc.z += t + e + fmaf(v.y, w.w, v.w * w.y);
  // im += v.re * w.im
  p = v.x * w.y; e = fmaf(v.x, w.y, -p);
  two_sum(acc.y, p, s, t); acc.y = s;
  acc.w += t + e + fmaf(v.x, w.w, v.z * w.y);
  // im -= v.im * w.re
  p = v.y * w.x; e = fmaf(v.y, w.x, -p);
  two_sum(acc.y, -p, s, t); acc.y = s;
  acc.w += t - e - fmaf(v.y, w.z, v.w * w.x);
}

// a += b for two accumulators in the convention above (FP32 operations only)
__device__ __forceinline__ void df_acc_add(float4& a, float4 b) {
  float s, t;
  two_sum(a.x, b.x, s, t);
  a.x = s;
  a.z += t + b.z;
  two_sum(a.y, b.y, s, t);
  a.y = s;
  a.w += t + b.w;
}

// Sum of an accumulator over the 32 lanes of a warp, in lane 0.
__device__ __forceinline__ float4 df_warp_sum(float4 v) {
  for (int off = 16; off > 0; off >>= 1) {
    float4 o;
    o.x = __shfl_down_sync(0xffffffffu, v.x, off);
    o.y = __shfl_down_sync(0xffffffffu, v.y, off);
    o.z = __shfl_down_sync(0xffffffffu, v.z, off);
    o.w = __shfl_down_sync(0xffffffffu, v.w, off);
    df_acc_add(v, o);
  }
  return v;
}

// ---- normalised double-float reals (hi, lo with |lo| <= ulp(hi) / 2) and complex values
struct dd {
  float hi, lo;
};
struct cdd {
  dd re, im;
};

__device__ __forceinline__ dd dd_norm(float s, float t) {
  const float hi = s + t;
  return dd{hi, t - (hi - s)};
}
__device__ __forceinline__ dd dd_make(double v) {
  const float hi = __double2float_rn(v);
  return dd{hi, __double2float_rn(v - (double)hi)};
}

// ---- FP64 <-> double-float without FP64 instructions.  GB300 retires FP64 arithmetic and
// the FP64 <-> FP32 conversions at about the FP64 rate (1/64 of FP32), so streaming
// kernels convert with integer operations on the IEEE 754 bit patterns (binary64: sign,
// 11 exponent bits with bias 1023, 52 fraction bits; binary32: sign, 8 with bias 127, 23).

// (double)f exactly: exponent rebiased by 1023 - 127 = 896, fraction moved to the top of
// the 52-bit field.  Subnormals, infinities and NaNs take the conversion instruction.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u || e == 0xFFu) {
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)sgn);   // signed zero
    return (double)f;
  }
  return __longlong_as_double(
      (long long)(sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// x = hi + lo + d, |d| < 2^-46 |x|: hi holds the leading 24 significand bits of x
// (truncated), lo the next 23 (truncated); 0 <= lo / hi < ulp(hi) / hi, so the pair is
// not normalised in the round-to-nearest sense, which the operations below allow.
// Zeros are exact; |x| outside [2^-103, 2^128) takes the conversion instructions.
__device__ __forceinline__ dd split_d(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(u >> 32) & 0x80000000u;
  const int fe = (int)((u >> 52) & 0x7FFu) - 896;   // biased binary32 exponent of x
  if (fe < 24 || fe > 254) {
    if ((u << 1) == 0ull) return dd{__uint_as_float(sgn), 0.f};
    return dd_make(x);
  }
  const float hi = __uint_as_float(sgn | ((unsigned)fe << 23) | ((unsigned)(u >> 29) & 0x7FFFFFu));
  // fraction bits 28..6 below hi as r * 2^-23 in [0, 1) (exact), then scaled by their
  // weight 2^(fe - 150), a normal float for fe >= 24; the product is exact
  const float f = __uint_as_float(0x3F800000u | ((unsigned)(u >> 6) & 0x7FFFFFu)) - 1.0f;
  const float lo = f * __uint_as_float((unsigned)(fe - 23) << 23);
  return dd{hi, __uint_as_float(__float_as_uint(lo) | sgn)};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  return dd_norm(s, t + a.lo + b.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p) + fmaf(a.hi, b.lo, a.lo * b.hi);
  return dd_norm(p, e);
}
// a * b with b an exact float
__device__ __forceinline__ dd dd_mulf(dd a, float b) {
  const float p = a.hi * b;
  return dd_norm(p, fmaf(a.hi, b, -p) + a.lo * b);
}
__device__ __forceinline__ dd dd_prodf(float a, float b) {
  const float p = a * b;
  return dd_norm(p, fmaf(a, b, -p));
}

__device__ __forceinline__ cdd cdd_load(float4 v) { return cdd{dd{v.x, v.z}, dd{v.y, v.w}}; }
__device__ __forceinline__ float4 cdd_store(cdd a) { return make_float4(a.re.hi, a.im.hi, a.re.lo, a.im.lo); }
__device__ __forceinline__ cdd cdd_make(double2 v) { return cdd{dd_make(v.x), dd_make(v.y)}; }
__device__ __forceinline__ cdd cdd_add(cdd a, cdd b) { return cdd{dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ cdd cdd_sub(cdd a, cdd b) {
  return cdd{dd_add(a.re, dd_neg(b.re)), dd_add(a.im, dd_neg(b.im))};
}
__device__ __forceinline__ cdd cdd_mul(cdd a, cdd b) {
  return cdd{dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im))),
             dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
// a * z with z a complex of exact floats
__device__ __forceinline__ cdd cdd_mulf(cdd a, float2 z) {
  return cdd{dd_add(dd_mulf(a.re, z.x), dd_neg(dd_mulf(a.im, z.y))),
             dd_add(dd_mulf(a.re, z.y), dd_mulf(a.im, z.x))};
}
__device__ __forceinline__ cdd cdd_scale(cdd a, dd s) { return cdd{dd_mul(a.re, s), dd_mul(a.im, s)}; }
// w * z with w a small exact float weight and z a complex of exact floats
__device__ __forceinline__ cdd cdd_wz(float w, float2 z) { return cdd{dd_prodf(w, z.x), dd_prodf(w, z.y)}; }
__device__ __forceinline__ cdd cdd_zero() { return cdd{dd{0.f, 0.f}, dd{0.f, 0.f}}; }

// ---- running accumulators: the high part is carried by Knuth's two-sum, the rounding
// errors of sums and of Dekker products collect in the low part, and the sum is
// normalised once, where it leaves the accumulator.
struct racc {
  float hi, lo;
};
__device__ __forceinline__ void racc_add(racc& a, float t) {   // + t, t an exact float
  float s, e;
  two_sum(a.hi, t, s, e);
  a.hi = s;
  a.lo += e;
}
__device__ __forceinline__ void racc_add_prod(racc& a, float x, float y) {   // + x y
  const float p = x * y;
  const float pe = fmaf(x, y, -p);
  float s, e;
  two_sum(a.hi, p, s, e);
  a.hi = s;
  a.lo += e + pe;
}
__device__ __forceinline__ void racc_add_ddf(racc& a, dd x, float y) {   // + x y, y an exact float
  const float p = x.hi * y;
  const float pe = fmaf(x.hi, y, -p) + x.lo * y;
  float s, e;
  two_sum(a.hi, p, s, e);
  a.hi = s;
  a.lo += e + pe;
}
__device__ __forceinline__ void racc_add_dd(racc& a, dd x, dd y) {   // + x y (y may be unnormalised)
  const float p = x.hi * y.hi;
  const float pe = fmaf(x.hi, y.hi, -p) + fmaf(x.hi, y.lo, x.lo * y.hi);
  float s, e;
  two_sum(a.hi, p, s, e);
  a.hi = s;
  a.lo += e + pe;
}
__device__ __forceinline__ dd racc_dd(racc a) { return dd_norm(a.hi, a.lo); }
__device__ __forceinline__ dd dd_of(racc a) { return dd{a.hi, a.lo}; }
// a += x z for a double-float complex x and a complex z of exact floats (sign s = +-1)
__device__ __forceinline__ void cacc_add_cz(racc& re, racc& im, cdd x, float2 z, float s) {
  racc_add_ddf(re, x.re, s * z.x);
  racc_add_ddf(re, x.im, -s * z.y);
  racc_add_ddf(im, x.re, s * z.y);
  racc_add_ddf(im, x.im, s * z.x);
}

// a -= h v for double-float complex h and v (re, im accumulators)
__device__ __forceinline__ void cacc_sub_cdd(racc& re, racc& im, cdd h, cdd v) {
  racc_add_dd(re, dd_neg(h.re), v.re);
  racc_add_dd(re, h.im, v.im);
  racc_add_dd(im, dd_neg(h.re), v.im);
  racc_add_dd(im, dd_neg(h.im), v.re);
}

}  // namespace helm

// Double-float arithmetic on the FP32 pipes, shared by the transforms and the
// combine pass: a value is an unevaluated sum hi + lo of two FP32 numbers
// (about 48 significant bits); error-free transformations after Knuth
// (TwoSum), Dekker (FastTwoSum) and the FMA form of TwoProduct.  A complex
// value is a float4 (re_hi, re_lo, im_hi, im_lo).
#pragma once

#include <cuda_runtime.h>

namespace rexi {

__device__ __forceinline__ float2 f_fast(float s, float e) {
  const float h = s + e;
  return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float2 f_add(float a, float al, float b, float bl) {
  const float s = a + b, bb = s - a;
  return f_fast(s, ((a - (s - bb)) + (b - bb)) + (al + bl));
}
// x * y for double-floats x = (a, al), y = (b, bl), as an unnormalised pair
__device__ __forceinline__ float2 f_mul(float a, float al, float b, float bl) {
  const float p = a * b;
  return make_float2(p, fmaf(a, bl, fmaf(al, b, fmaf(a, b, -p))));
}
__device__ __forceinline__ float4 cadd(float4 a, float4 b) {
  const float2 r = f_add(a.x, a.y, b.x, b.y), i = f_add(a.z, a.w, b.z, b.w);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ float4 csub(float4 a, float4 b) {
  const float2 r = f_add(a.x, a.y, -b.x, -b.y), i = f_add(a.z, a.w, -b.z, -b.w);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ float4 cmul(float4 a, float4 w) {
  const float2 rr = f_mul(a.x, a.y, w.x, w.y), ii = f_mul(a.z, a.w, w.z, w.w);
  const float2 ri = f_mul(a.x, a.y, w.z, w.w), ir = f_mul(a.z, a.w, w.x, w.y);
  const float2 re = f_add(rr.x, rr.y, -ii.x, -ii.y), im = f_add(ri.x, ri.y, ir.x, ir.y);
  return make_float4(re.x, re.y, im.x, im.y);
}
// real double-float times complex double-float
__device__ __forceinline__ float4 crmul(float2 a, float4 w) {
  const float2 re = f_mul(a.x, a.y, w.x, w.y), im = f_mul(a.x, a.y, w.z, w.w);
  const float2 r = f_fast(re.x, re.y), i = f_fast(im.x, im.y);
  return make_float4(r.x, r.y, i.x, i.y);
}
__device__ __forceinline__ float2 f_mulf(float2 a, float2 b) {
  const float2 p = f_mul(a.x, a.y, b.x, b.y);
  return f_fast(p.x, p.y);
}
__device__ __forceinline__ float2 f_addf(float2 a, float2 b) { return f_add(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 f_subf(float2 a, float2 b) { return f_add(a.x, a.y, -b.x, -b.y); }
__device__ __forceinline__ float4 cconj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }

// FP64 <-> double-float at the HBM boundary without FP64 arithmetic (on this
// GPU an FP64 instruction, conversions included, costs about 30 FP32 ones).
// double -> (hi, lo): hi keeps the top 24 bits of the significand
// (truncated), lo the next 29 bits rounded to 24, both by integer operations;
// |v - (hi + lo)| <= 2^-47 |v|.  Used for zero and |v| in [2^-74, 2^127);
// other values take the FP64 route.
// The FP64 routes are out-of-line calls so that the compiler does not
// execute them under a predicate for every value.
static __device__ __noinline__ float2 df_from_double_fp64(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
static __device__ __noinline__ double widen_float_fp64(float f) { return (double)f; }

__device__ __forceinline__ float2 df_from_double(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b << 1) == 0ull) return make_float2(0.f, 0.f);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if (e < 949u || e > 1150u) return df_from_double_fp64(v);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long m = b & 0xfffffffffffffull;
  const float hi = __uint_as_float(sign | ((e - 896u) << 23) | (unsigned)(m >> 29));
  const float scale = __uint_as_float((e - 948u) << 23);  // 2^(e - 1075), a normal float here
  const float lo = __uint2float_rn((unsigned)(m & 0x1fffffffull)) * scale;
  return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sign));
}
// float -> double exactly by re-biasing the exponent (integer operations);
// zero, subnormals, infinities and NaN through the FP64 conversion.
__device__ __forceinline__ double widen_float(float f) {
  const unsigned u = __float_as_uint(f);
  if ((u << 1) == 0u) return __longlong_as_double((long long)((unsigned long long)(u >> 31) << 63));
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0u || ef == 255u) return widen_float_fp64(f);
  const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(ef + 896u) << 52) |
                                  ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)bits);
}
// (hi, lo) -> double: one FP64 addition.
__device__ __forceinline__ double df_to_double(float2 a) { return widen_float(a.x) + widen_float(a.y); }

}  // namespace rexi

// FP32 pairs ("float-float", a value is hi + lo): conversions from and to
// double with integer operations only (no FP64-pipe work), exact FMA
// two-products (Dekker) and two-sum accumulation (Knuth), ~2^-48 relative.
#pragma once
#include <cuda_runtime.h>

struct ffn {
  float hi, lo;
};

// Exact split of a double into an FP32 pair with integer operations only
// (no FP64-pipe conversions): hi keeps the top 24 significant bits, lo the
// next bits rounded to 24 (|d - hi - lo| <= 2^-47 |d|).  Values below 2^-74
// keep hi only; values outside the FP32 range saturate.
__device__ __forceinline__ ffn ff_split(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const int ef = e - 1023 + 127;
  if (ef <= 0) return ffn{0.0f, 0.0f};
  if (ef >= 255) return ffn{__uint_as_float(sign | 0x7F800000u), 0.0f};
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)(mant >> 29));
  float lo = 0.0f;
  const unsigned mlo = (unsigned)(mant & 0x1FFFFFFFu);
  if (mlo != 0u && e >= 949) {
    lo = __uint2float_rn(mlo) * __uint_as_float((unsigned)(e - 948) << 23);
    if (sign) lo = -lo;
  }
  return ffn{hi, lo};
}
// float -> double exactly, with integer operations
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xFF;
  if (ex == 0) return 0.0;  // zero (FP32 denormals do not occur here)
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ex - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}


// a + b for pairs (two-sum on the high parts, low parts added, renormalised)
__device__ __forceinline__ ffn ff_add(ffn a, ffn b) {
  float s = a.hi + b.hi;
  float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  float t = s + e;
  return ffn{t, e - (t - s)};
}
// acc += a * b: exact product of the high parts (FMA), cross terms in FP32,
// the high sum by two-sum; the low part collects all rounding errors
__device__ __forceinline__ void ff_acc_prod(ffn& acc, ffn a, ffn b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  acc.lo += ((acc.hi - (s - bb)) + (p - bb)) + e;
  acc.hi = s;
}
__device__ __forceinline__ ffn ff_negate(ffn a) { return ffn{-a.hi, -a.lo}; }
__device__ __forceinline__ ffn ff_sub(ffn a, ffn b) { return ff_add(a, ff_negate(b)); }
// c * d as an unnormalised pair: the exact product of the high parts (FMA)
// plus the cross terms (the lo * lo term is below the pair's precision)
__device__ __forceinline__ ffn ff_prod(ffn c, ffn d) {
  const float p = c.hi * d.hi;
  float e = fmaf(c.hi, d.hi, -p);
  e = fmaf(c.hi, d.lo, fmaf(c.lo, d.hi, e));
  return ffn{p, e};
}
// d * 2^-sh split into a pair (exponents shifted with integer operations, so
// the scaling is exact); doubles whose scaled value falls below the double
// range give zero
__device__ __forceinline__ ffn ff_split_scaled(double d, int sh) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return ffn{0.0f, 0.0f};
  const int es = e - sh;
  if (es <= 0) return ffn{0.0f, 0.0f};
  return ff_split(__longlong_as_double(b - ((long long)sh << 52)));
}
// float * 2^sh -> double exactly, with integer operations (zero below the
// double range)
__device__ __forceinline__ double f2d_exact_scaled(float f, int sh) {
  const unsigned u = __float_as_uint(f);
  const int ex = (int)((u >> 23) & 0xFF);
  if (ex == 0) return 0.0;
  const int E = ex - 127 + 1023 + sh;
  if (E <= 0) return 0.0;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) | ((unsigned long long)E << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double ff_to_d_scaled(ffn a, int sh) {
  return f2d_exact_scaled(a.hi, sh) + f2d_exact_scaled(a.lo, sh);
}
__device__ __forceinline__ double ff_to_d(ffn a) { return f2d_exact(a.hi) + f2d_exact(a.lo); }
__device__ __forceinline__ ffn ff_warp_sum(ffn x) {
  for (int o = 16; o > 0; o >>= 1) {
    ffn y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
    x = ff_add(x, y);
  }
  return x;
}

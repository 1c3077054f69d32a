// Pairs of binary32 values (hi + lo) as a ~48-bit floating-point format, for the binary64-accuracy
// parts of the path that would otherwise run on GB300's binary64 pipe (two FMA per SM and clock,
// against 128 binary32).  Built on the error-free transformations: the sum of two floats equals
// their rounded sum plus an error that is itself a float (Knuth's TwoSum), and the product of two
// floats equals the rounded product plus fma(a, b, -p) (the FMA form of Dekker's exact product).
// Every operation below uses round-to-nearest intrinsics so that no multiply is contracted into an
// addition and no sum is reassociated.
#pragma once

#include <stdint.h>

namespace hhg {

// s + e = a + b exactly, s = fl(a + b)
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// Running sum of pair-times-pair products: (hi, lo) with hi carrying the rounded total and lo the
// accumulated errors (|lo| stays a few units in the last place of hi; renormalise before use).
struct DfAcc {
  float hi = 0.f, lo = 0.f;
  // += (ah + al)(bh + bl), dropping al * bl (relative size 2^-48)
  __device__ __forceinline__ void add_prod(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);  // exact error of p
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float2 s = df_two_sum(hi, p);
    hi = s.x;
    lo = __fadd_rn(lo, __fadd_rn(s.y, e));
  }
  // += (ah + al)
  __device__ __forceinline__ void add(float2 a) {
    const float2 s = df_two_sum(hi, a.x);
    hi = s.x;
    lo = __fadd_rn(lo, __fadd_rn(s.y, a.y));
  }
  __device__ __forceinline__ float2 value() const { return df_fast_two_sum(hi, lo); }
};

// The conversion instructions between binary32 and binary64 run on GB300's binary64 pipe, so the
// common cases below use integer operations, and the rare ones call these (never inlined, so the
// compiler cannot evaluate them speculatively on every call).
static __device__ __noinline__ float2 df_split_slow(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
static __device__ __noinline__ double df_widen_slow(float f) { return (double)f; }

// binary32 -> binary64 exactly: exponent re-biased, significand shifted (zero and normal values;
// subnormals, infinities and NaN take the conversion instruction)
__device__ __forceinline__ double df_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sg = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u << 1) == 0u) return __longlong_as_double((long long)sg);
  if (ex == 0u || ex == 0xffu) return df_widen_slow(f);
  return __longlong_as_double(
      (long long)(sg | ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// Split a binary64 value into hi + lo, both binary32: hi is x with its significand cut to 24 bits,
// lo the next 24 bits of the rest (bits below are dropped: |x - hi - lo| < 2^-47 |x|).  Integer
// operations only for binary64 values whose hi is a normal binary32 (2^-126 <= |x| < 2^128); zero
// gives (0, 0); values outside that range take the rounding conversions (binary64 arithmetic).
__device__ __forceinline__ float2 df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned top = (unsigned)(b >> 32);
  const int e = (int)((top >> 20) & 0x7ffu);  // biased binary64 exponent
  const int eh = e - 1023 + 127;              // biased binary32 exponent of hi
  if (eh <= 0 || eh >= 255) {
    // zero (tested on the two 32-bit words: a comparison of x with 0.0 would be a binary64 instruction)
    if (((top & 0x7fffffffu) | (unsigned)b) == 0u) return make_float2(0.f, 0.f);
    return df_split_slow(x);
  }
  const unsigned sgn = top & 0x80000000u;
  const unsigned long long mant = b & 0xfffffffffffffull;  // 52 significand bits
  const float h = __uint_as_float(sgn | ((unsigned)eh << 23) | (unsigned)(mant >> 29));
  const unsigned r = (unsigned)(mant & 0x1fffffffull);  // the 29 bits below hi's significand
  if (r == 0u) return make_float2(h, 0.f);
  // r * 2^(e - 1075) as a binary32: leading bit at position p, 24 bits kept
  const int p = 31 - __clz(r);
  const int sh = p - 23;
  const unsigned m24 = sh >= 0 ? (r >> sh) : (r << -sh);
  const int el = sh + e - 925;  // biased binary32 exponent of lo
  if (el <= 0) return make_float2(h, 0.f);  // |lo| < 2^-126: below binary32's normal range
  return make_float2(h, __uint_as_float(sgn | ((unsigned)el << 23) | (m24 & 0x7fffffu)));
}

// hi + lo in binary64 (one binary64 addition; exact when the pair came from df_split)
__device__ __forceinline__ double df_to_double(float2 a) { return df_widen(a.x) + df_widen(a.y); }

}  // namespace hhg

// float-float ("double-float") arithmetic on the float32 pipe.
//
// GB300 executes float64 arithmetic (and float64<->float32 conversion) at ~1/70 of the
// float32 rate, so the refinement keeps its iterate and evaluates its residual as
// unevaluated sums hi + lo of two floats (~48-bit significand).  The building blocks
// are the error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the
// fused multiply-add product error; conversions from and to float64 work on the bit
// patterns with integer instructions only.
#pragma once
#include <cstdint>

namespace sp {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float h) { return ff{h, 0.f}; }

// s + e = a + b exactly.  The _rn intrinsics keep the compiler from contracting a
// product into these sums, which would break the error-free transformations.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) {
  float s, e;
  two_sum(a.hi, -b.hi, s, e);
  e += a.lo - b.lo;
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// Split a float64 into hi + lo floats using integer operations only: hi is x rounded to
// the nearest float (ties away from zero), lo the remainder rounded to float, so
// |hi + lo - x| <= 2^-48 |x|.  Magnitudes below 2^-126 flush to zero; above float range
// saturate to infinity.
__device__ __forceinline__ ff d2ff(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int whi = (unsigned int)(b >> 32);
  const unsigned int wlo = (unsigned int)b;
  const unsigned int sgn = whi & 0x80000000u;
  const int e = (int)((whi >> 20) & 0x7FFu);
  int E = e - 1023;
  if (e == 0 || E < -126) return ff{0.f, 0.f};
  unsigned int t = ((whi & 0xFFFFFu) << 3) | (wlo >> 29);
  int rem = (int)(wlo & 0x1FFFFFFFu);
  if (rem >= 0x10000000) {
    t += 1u;
    rem -= 0x20000000;
  }
  if (t == 0x800000u) {
    t = 0u;
    E += 1;
  }
  if (E > 127) return ff{__uint_as_float(sgn | 0x7F800000u), 0.f};
  const float hi = __uint_as_float(sgn | ((unsigned int)(E + 127) << 23) | t);
  const int sh = E - 52;   // lo = rem * 2^sh, applied as two exact power-of-two scalings
  const int s1 = sh / 2, s2 = sh - s1;
  float lo = (float)rem * __uint_as_float((unsigned int)(s1 + 127) << 23) * __uint_as_float((unsigned int)(s2 + 127) << 23);
  return ff{hi, sgn ? -lo : lo};
}

// Exact float -> float64 through the bit pattern (normal numbers and zero; denormals
// flush to zero, infinities and NaN keep their class).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double((long long)s);
  unsigned long long ed = (e == 0xFFu) ? 0x7FFull : (unsigned long long)(e - 127u + 1023u);
  const unsigned long long bits = s | (ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// float64 value of hi + lo (one float64 addition).
__device__ __forceinline__ double ff2d(ff a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace sp

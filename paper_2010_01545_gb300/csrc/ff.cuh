// ff.cuh -- "double-float" arithmetic: a binary64 value carried as an
// unevaluated sum hi + lo of two binary32 numbers, computed on the binary32
// pipes (74x the binary64 rate on GB300).
//
// Algorithms: Knuth's TwoSum and FMA-based TwoProduct (error-free
// transformations), Dekker's Fast2Sum for renormalisation.  Sums are TwoSum
// of the high parts with the low parts added in binary32; products are the
// exact product of the high parts plus the two cross terms.  Neither is
// renormalised: the low part of every intermediate stays below about 2^-22
// times the magnitude of the operands it came from (after cancellation the
// high part may be much smaller than that), so each rounding error is about
// 2^-47 of the operands' magnitudes, which is the scale the normwise error of
// the stencil is measured on.  The result is renormalised once, when it is
// assembled into a double.  For the PW stencil, whose terms are at most a few
// times the largest source term, the normwise error against binary64 is
// about 1e-14 (the tests bound it by 1e-12).
//
// Splitting a double into (hi, lo) never touches the binary64 pipe (a dozen
// integer bit operations and one binary32 subtraction); assembling (hi, lo)
// into a double is either the same kind of integer sequence (truncating) or
// two conversions and one add on the otherwise idle binary64 pipe
// (to_double_fp64, rounding to nearest).  Range:
// magnitudes in [2^-80, 2^126]; smaller inputs lose relative precision (the
// low part underflows), zero is exact, and non-finite inputs are not
// supported.
#pragma once

#include <stdint.h>

namespace advect {

struct ff {
  float hi, lo;
  __device__ __forceinline__ ff() {}
  __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ ff(int z) : hi((float)z), lo(0.f) {}  // C(0)
  __device__ __forceinline__ explicit ff(double x);
  __device__ __forceinline__ explicit operator double() const;
};

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return ff(s, b - (s - a));
}

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ ff operator+(const ff& x, const ff& y) {
  const ff s = two_sum(x.hi, y.hi);
  return ff(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ ff operator-(const ff& x) { return ff(-x.hi, -x.lo); }
__device__ __forceinline__ ff operator-(const ff& x, const ff& y) { return x + (-y); }

__device__ __forceinline__ ff operator*(const ff& x, const ff& y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return ff(p, e);
}

__device__ __forceinline__ ff& operator+=(ff& x, const ff& y) { return x = x + y; }
__device__ __forceinline__ ff& operator-=(ff& x, const ff& y) { return x = x - y; }

// double -> (hi, lo): hi is x with its significand truncated to 24 bits
// (exact in binary32); lo holds the next 23 bits of the remainder.
//   hi: the top word with its exponent rebiased from 1023 to 127, funnel-
//       shifted left by 3 to take the first 3 bits of the low word, sign
//       put back;
//   lo: the 23 remainder bits placed under the exponent of 2^(e-23) minus
//       2^(e-23) itself -- an exact binary32 subtraction giving rem*2^(e-46).
// Zero and magnitudes below 2^-104 give (+-0, 0); below 2^-80 lo may be
// subnormal (and is dropped by the assembly below).
__device__ __forceinline__ ff::ff(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t top = (uint32_t)(b >> 32), bot = (uint32_t)b;
  const uint32_t sign = top & 0x80000000u;
  const uint32_t mag = __funnelshift_l(bot, top - 0x38000000u, 3) & 0x7fffffffu;
  const uint32_t base = (mag & 0x7f800000u) - 0x0b800000u;  // 2^(e-23)
  const uint32_t rem = (bot >> 6) & 0x7fffffu;
  const float l = __uint_as_float(base | rem) - __uint_as_float(base);
  const bool tiny = (top & 0x7fffffffu) < 0x39700000u;
  hi = __uint_as_float(tiny ? sign : (mag | sign));
  lo = tiny ? 0.f : __uint_as_float(__float_as_uint(l) | sign);
}

// (hi, lo) -> double: renormalise, then add lo into hi's binary64 pattern as
// an integer multiple of hi's binary64 ulp (truncated).  After the
// renormalisation |lo| <= ulp32(hi)/2, so that multiple fits in 29 bits.
__device__ __forceinline__ ff::operator double() const {
  // |hi| >= |lo| is not guaranteed after unnormalised arithmetic: order them
  const ff n = fabsf(hi) >= fabsf(lo) ? fast_two_sum(hi, lo) : fast_two_sum(lo, hi);
  const uint32_t hb = __float_as_uint(n.hi), lb = __float_as_uint(n.lo);
  const uint32_t mag = hb & 0x7fffffffu;
  const uint32_t dh = ((mag >> 3) + 0x38000000u) | (hb & 0x80000000u);  // exponent 127 -> 1023
  const uint32_t dl = hb << 29;
  const int sh = (int)((lb >> 23) & 0xffu) - (int)(mag >> 23) + 29;  // lo / ulp64(hi) = ml * 2^sh
  const uint32_t ml = (lb & 0x7fffffu) | 0x800000u;
  uint32_t L = sh >= 0 ? ml << sh : __funnelshift_rc(ml, 0u, (uint32_t)(-sh));
  L = (lb & 0x7f800000u) == 0 ? 0u : L;  // lo zero (or below the binary32 normal range)
  const bool opposite = ((hb ^ lb) & 0x80000000u) != 0;
  L = (opposite && (hb & 0x7fffffu) == 0) ? L << 1 : L;  // hi a power of two: the binade below
  const long long sL = opposite ? -(long long)L : (long long)L;
  const unsigned long long r = (((unsigned long long)dh << 32) | dl) + (unsigned long long)sL;
  return (mag >> 23) == 0 ? 0.0 : __longlong_as_double((long long)r);  // zero (binary32 subnormals as zero)
}

// (hi, lo) -> double on the binary64 pipe: both parts are exact in binary64
// and their sum is exact or rounded once to nearest, so the result is at least
// as close as the truncated assembly above.  Two conversions and one add per
// value, on a pipe the double-float arithmetic otherwise leaves idle; the
// forward sweep stores with it (measured 45.0 -> 47.9 Gpts/s at 2048 x 2048
// x 64), the adjoint keeps the integer assembly (it ran 6 % slower with this).
__device__ __forceinline__ double to_double_fp64(const ff& v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ ff shfl_up(const ff& v, int d) {
  return ff(__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d));
}
__device__ __forceinline__ ff shfl_down(const ff& v, int d) {
  return ff(__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d));
}

// Storage tag: binary64 in memory, double-float arithmetic.
struct f64ff {
  double v;
};

}  // namespace advect

// rt_filter.cuh -- cheap, rigorous bounds that let the argmin skip exact divisions.
//
// The waiting time of Eq. 25 is w = fl((P - T) / a).  Computing it costs a
// binary64 subtraction and division, which on GB300 occupy the FP64 pipe for
// about nine issue slots.  Most channels cannot be the minimum, and that can be
// shown with single-precision arithmetic: truncating the high 32-bit word of a
// non-negative double to a float (integer ops only, no FP64 conversion) gives a
// lower bound; adding one unit in the 20th mantissa bit gives an upper bound;
// float operations with directed rounding then give a certified lower bound of
// (P - T) and an upper bound of t * a.  A channel is skipped only if
//   (P - T)_lower > (t * a)_upper,  i.e.  its exact quotient exceeds t,
// so the exact minimum (with smallest-index ties) is unchanged.
#pragma once
#include <cstdint>

namespace rt {

// Float bounds from the high word hi of a non-negative double: the float with the
// same exponent and the top 20 fraction bits is hi * 8 - 0xC0000000 (mod 2^32) when
// the exponent is in the float's normal range (the exponent field moves from bit 20
// to bit 23 and is re-biased by 1023 - 127 = 896; 896 * 2^23 = 0xC0000000 mod 2^32).

// largest float <= x for a double x >= 0 (0 below FLT_MIN, just under FLT_MAX above it)
__device__ __forceinline__ float f32_lower(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x);
  const uint32_t h = min(hi, 0x47EFFFFFu);  // exponent field 1150: the float range's top
  return hi < (897u << 20) ? 0.0f : __uint_as_float(h * 8u - 0xC0000000u);
}

// a float >= x for a double x >= 0 (FLT_MIN below it, +inf above FLT_MAX)
__device__ __forceinline__ float f32_upper(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x);
  const uint32_t f = (max(hi, 897u << 20) * 8u - 0xC0000000u) + 8u;  // + one 2^-20 unit
  return hi >= (1151u << 20) ? __int_as_float(0x7F800000) : __uint_as_float(f);
}

// A float upper bound of the waiting time w = fl(fl(P - T) / a) of Eq. 25 (a > 0, T >= 0):
// an upper bound of P - T over a lower bound of a, divided with __fdividef (documented: at
// most 2 ulp from the rounded quotient for divisors in [2^-126, 2^126]) and widened by
// 2^-18, which also covers the two binary64 roundings; +inf for divisors outside that range.
// 0 when P - T is certainly <= 0 (then w = 0).
__device__ __forceinline__ float quot_upper(double P, double T, double a) {
  const float rem = __fsub_ru(f32_upper(P), f32_lower(T));
  if (!(rem > 0.0f)) return 0.0f;
  const float alo = f32_lower(a);
  if (!(alo >= 0x1p-125f) || alo > 0x1p125f) return __int_as_float(0x7F800000);
  return __fmul_ru(__fdividef(rem, alo), 1.000003814697265625f);  // 1 + 2^-18
}

// The next float above a finite x >= 0 (+inf stays +inf).
__device__ __forceinline__ float f32_next_up(float x) {
  return x < __int_as_float(0x7F800000) ? __int_as_float(__float_as_int(x) + 1) : x;
}

// True if the exact (P - T) / a is certainly > thr (a > 0, T >= 0, thr >= 0).
__device__ __forceinline__ bool exceeds(double P, double T, double a, float thr) {
  const float rem_lo = __fsub_rd(f32_lower(P), f32_upper(T));
  return rem_lo > __fmul_ru(thr, f32_upper(a));
}

}  // namespace rt

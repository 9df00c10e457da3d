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

// True if the exact (P - T) / a is certainly > thr (a > 0, T >= 0, thr >= 0).
__device__ __forceinline__ bool exceeds(double P, double T, double a, float thr) {
  const float rem_lo = __fsub_rd(f32_lower(P), f32_upper(T));
  return rem_lo > __fmul_ru(thr, f32_upper(a));
}

}  // namespace rt

// rt_sim.cuh -- per-event building blocks shared by the simulation kernels.
//
// Floating-point rules (so every mapping reproduces the same bits): each
// operation is one explicitly rounded binary64 op (__dadd_rn, __dsub_rn,
// __dmul_rn, __ddiv_rn; never contracted into an FMA).  Comparisons of values
// known to be non-negative (times, waiting times, propensities) are done on
// their bit patterns as signed 64-bit integers, which orders them exactly like
// the doubles and keeps the comparison off GB300's narrow FP64 pipe.
#pragma once
#include <cstdint>

#include "rt_filter.cuh"
#include "rt_internal.h"
#include "rt_rng.cuh"

namespace rt {

__device__ __forceinline__ int64_t dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd(int64_t b) { return __longlong_as_double(b); }
constexpr int64_t kInfBits = 0x7FF0000000000000ll;

// Exact binary64 value of 0 <= h < 2^53 built with integer instructions (the
// hardware int64 -> double conversion issues on the FP64 pipe); larger h rounds
// through the hardware conversion.
__device__ __forceinline__ double i64_to_f64(int64_t h) {
  if (h <= 0) return h == 0 ? 0.0 : __ll2double_rn(h);
  if (h >= (1ll << 53)) return __ll2double_rn(h);
  const int e = 63 - __clzll(h);  // position of the leading one, <= 52
  const uint64_t mant = (uint64_t)h << (52 - e);
  return __longlong_as_double((long long)((((uint64_t)(e + 1023)) << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
}

// c * h rounded to nearest-even for a finite c >= 0 and an integer 0 <= h < 2^32,
// with integer instructions: the 85-bit product of c's significand and h is rounded
// to 53 bits.  Other operands, and products outside the normal range, use the
// FP64 pipe (identical result: h is exact in binary64).
__device__ __forceinline__ double mul_rn_pos_u32(double c, int64_t h) {
  if (h == 0) return 0.0;  // c is finite and >= 0
  const uint64_t bc = (uint64_t)__double_as_longlong(c);
  const int ec = (int)(bc >> 52);
  if (h < 0 || h >= (1ll << 32) || ec == 0 || ec >= 0x7FF) return __dmul_rn(c, i64_to_f64(h));
  const uint64_t cm = (bc & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  const uint64_t a0 = (uint64_t)(uint32_t)cm * (uint32_t)h;          // low limb product
  const uint64_t a1 = (uint64_t)(uint32_t)(cm >> 32) * (uint32_t)h;  // high limb product (< 2^53)
  const uint64_t lo = a0 + (a1 << 32);
  const uint64_t hi = (a1 >> 32) + (lo < a0 ? 1u : 0u);  // product = hi 2^64 + lo, < 2^85
  const int len = hi ? 128 - __clzll(hi) : 64 - __clzll(lo);  // bit length, 53..85
  const int sh = len - 53;                                    // 0..32
  if (sh == 0) return __longlong_as_double((long long)(((uint64_t)ec << 52) | (lo & 0x000FFFFFFFFFFFFFull)));
  uint64_t m = (lo >> sh) | (hi << (64 - sh));
  const uint64_t rest = lo & ((1ull << sh) - 1), half = 1ull << (sh - 1);
  m += (rest > half || (rest == half && (m & 1))) ? 1 : 0;
  int e = ec + sh;
  if (m >> 53) {
    m >>= 1;
    e += 1;
  }
  if (e >= 0x7FF) return __dmul_rn(c, i64_to_f64(h));
  return __longlong_as_double((long long)(((uint64_t)e << 52) | (m & 0x000FFFFFFFFFFFFFull)));
}

// h_k(X) of Eq. 2 for a descriptor {s0, s1}, exact in int64, then a_k = c_k h_k (Eq. 1).
// IMUL: the product on integer instructions (faster where the FP64 pipe is the
// bottleneck) or on the FP64 pipe (the large-network scan, where the integer code
// in its loop costs more than it saves); both give the same bits.
template <bool IMUL = true, typename XAt>
__device__ __forceinline__ double propensity(int2 rd, double c, XAt x) {
  int64_t h;
  if (rd.x < 0) {
    h = 1;
  } else {
    const int64_t x0 = x(rd.x);
    if (rd.y == RD_UNI) h = x0;
    else if (rd.y == RD_DIMER) h = x0 * (x0 - 1) / 2;
    else h = x0 * (int64_t)x(rd.y);
  }
  return IMUL ? mul_rn_pos_u32(c, h) : __dmul_rn(c, i64_to_f64(h));
}

// Waiting time (P - T) / a of Eq. 25 for a > 0: 0 if no internal time is left.
__device__ __forceinline__ double waiting_time(double P, double T, double a) {
  const double rem = __dsub_rn(P, T);
  return dbits(rem) > 0 ? __ddiv_rn(rem, a) : 0.0;
}

// Time-dependent rates c_k(t) = c_k (1 + beta_k t) (Sec. 6, Eq. 29): with A = c_k h_k(X)
// constant between events, the waiting time d solving A (d (1 + beta t) + beta d^2 / 2) = R
// for the remaining internal time R = P - T (the positive root, written without cancellation),
// and the integral of 1 + beta s over [t, t + d].  beta = 0 gives the constant-rate operations.
__device__ __forceinline__ double tdep_wait(double A, double beta, double R, double t) {
  if (!(dbits(R) > 0)) return 0.0;
  if (beta == 0.0) return __ddiv_rn(R, A);
  const double u = __dadd_rn(1.0, __dmul_rn(beta, t));
  const double b = __dmul_rn(A, u);
  const double e = __dmul_rn(__dmul_rn(__dmul_rn(2.0, A), beta), R);
  const double den = __dadd_rn(b, __dsqrt_rn(__dadd_rn(__dmul_rn(b, b), e)));
  return __ddiv_rn(__dmul_rn(2.0, R), den);
}

__device__ __forceinline__ double tdep_integral(double beta, double t, double d) {
  if (beta == 0.0) return d;
  const double u = __dadd_rn(1.0, __dmul_rn(beta, t));
  return __dadd_rn(__dmul_rn(d, u), __dmul_rn(__dmul_rn(__dmul_rn(beta, d), d), 0.5));
}

// The same from an already computed remainder rem = fl(P - T).
__device__ __forceinline__ double waiting_time_rem(double rem, double a) {
  return dbits(rem) > 0 ? __ddiv_rn(rem, a) : 0.0;
}

// An estimate of the quotient rem / a (rem > 0, a > 0) used only to pick which
// channel to compute exactly first; the exclusion test below is what is rigorous.
__device__ __forceinline__ float quot_estimate(double rem, double a) {
  return __fdividef(f32_upper(rem), f32_lower(a) + 1e-37f);
}

// True if the exact quotient rem / a is certainly > thr (rem > 0, a > 0).
__device__ __forceinline__ bool quot_exceeds(double rem, double a, float thr) {
  return f32_lower(rem) > __fmul_ru(thr, f32_upper(a));
}

// An estimate of (P - T) / a used only to choose the candidate that is computed
// exactly first (any choice gives the same, exact result).
__device__ __forceinline__ float wait_estimate(double P, double T, double a) {
  const float rem = f32_upper(P) - f32_lower(T);
  return rem > 0.0f ? __fdividef(rem, f32_lower(a) + 1e-37f) : 0.0f;
}

// Per-event trace: event ev of trajectory j fired channel mu at time t (recorded for
// the first trace_len events).
__device__ __forceinline__ void trace_event(const rt_outputs &o, int64_t j, int32_t ev, int mu, double t) {
  if (ev < o.trace_len) {
    if (o.trace_mu_dev) o.trace_mu_dev[j * o.trace_len + ev] = mu;
    if (o.trace_t_dev) o.trace_t_dev[j * o.trace_len + ev] = t;
  }
}

// The unused rest of trajectory j's trace, entries [ev, trace_len): -1 and 0, written
// by nthr cooperating threads (this one is number tid).
__device__ __forceinline__ void trace_tail(const rt_outputs &o, int64_t j, int32_t ev, int tid, int nthr) {
  for (int64_t e = (int64_t)ev + tid; e < o.trace_len; e += nthr) {
    if (o.trace_mu_dev) o.trace_mu_dev[j * o.trace_len + e] = -1;
    if (o.trace_t_dev) o.trace_t_dev[j * o.trace_len + e] = 0.0;
  }
}

// Register-array element r (runtime) by predicated selects, so arrays indexed with
// compile-time indices stay in registers.
template <int R, typename T>
__device__ __forceinline__ T pick(const T (&v)[R], int r) {
  T out = v[0];
#pragma unroll
  for (int i = 1; i < R; ++i) out = (i == r) ? v[i] : out;
  return out;
}

}  // namespace rt

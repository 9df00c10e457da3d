// rt_rng.cuh -- device random draws for the random time algorithm.
//
// Eq. 24 of Liu & Wang (arXiv:2103.00405): each channel's internal-time
// increment is ln(1/r) with r uniform, i.e. Exp(1).  The uniform comes from
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by the seed and
// indexed by (draw index >> 1, trajectory, channel, stream), so every channel is
// its own unit-rate Poisson process Y_k of Eq. 16 and any draw can be
// recomputed without state.
//
// The logarithm uses only integer instructions (GB300 issues 32-bit integer
// work at roughly fifty times its FP64 rate) and rounds once to binary64:
//   ln(M 2^E) = (E + q) ln2 + ln(m),  m = M / 2^q in [sqrt(1/2), sqrt(2)),
//   ln(m) = 2 atanh(s), s = (m - 1)/(m + 1), 2 atanh(s) = 2 s (1 + sum_i s^2i/(2i+1)),
// with s held in 64-bit fixed point (the quotient is the exact floor), the
// series to i = 12 by Horner's rule in Q64 (truncating products), ln2 as
// round(ln2 * 2^64), and a 128-bit fixed-point sum rounded to nearest-even.
#pragma once
#include <cstdint>

namespace rt {

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Philox4x32-10
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// 64 random bits of draw `n` of channel k in trajectory g.
__device__ __forceinline__ uint64_t draw_bits(uint64_t seed, uint64_t g, uint32_t k, uint32_t n, uint32_t stream) {
  const uint4 o = philox4x32_10(make_uint4(n >> 1, (uint32_t)g, k, stream), (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t w0 = (n & 1u) ? o.z : o.x;
  const uint32_t w1 = (n & 1u) ? o.w : o.y;
  return ((uint64_t)w1 << 32) | w0;
}

// ---------------------------------------------------------------------------
// 128-bit helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int clz128(u128 v) {
  const uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
  return hi ? __clzll(hi) : 64 + __clzll(lo);
}

// Nearest binary64 to V * 2^scale (V > 0), ties to even; result known to be normal.
__device__ __forceinline__ double round_to_f64(u128 V, int scale) {
  const int p = 127 - clz128(V);
  uint64_t mant;
  int e = p;
  if (p <= 52) {
    mant = (uint64_t)V << (52 - p);
  } else {
    const int sh = p - 52;
    uint64_t q = (uint64_t)(V >> sh);
    const u128 rem = V & (((u128)1 << sh) - 1);
    const u128 half = (u128)1 << (sh - 1);
    q += (rem > half || (rem == half && (q & 1))) ? 1 : 0;
    if (q >> 53) {
      q >>= 1;
      e += 1;
    }
    mant = q;
  }
  const uint64_t bits = ((uint64_t)(e + scale + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// floor(n * 2^63 / d) for n, d in [2^63, 2^64).  x = 2^64 + v approximates
// 2^128 / d from below: a float reciprocal of d rounded up, itself rounded toward
// zero, then two Newton steps x += x (2^128 - d x) / 2^128 with truncated
// products.  Newton's reciprocal iteration started below the root stays below it
// and increases, so v never wraps; the quotient estimate is then at most a few
// units low and is made exact by comparing the remainder with d.
__device__ __forceinline__ uint64_t quot_q63(uint64_t n, uint64_t d) {
  const float r = __frcp_rz((float)((uint32_t)(d >> 40) + 1u));  // <= 2^40 / d, in [2^-24, 2^-23)
  const uint64_t R = __float2ull_rz(r * 0x1p62f);                 // in [2^38, 2^39)
  uint64_t v = (R - (1ull << 38)) << 26;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const u128 dx = ((u128)d << 64) + (u128)d * v;
    const uint64_t ehi = (uint64_t)((((u128)0) - dx) >> 64);  // (2^128 - d x) / 2^64 >= 0
    v += ehi + __umul64hi(v, ehi);
  }
  uint64_t q = (uint64_t)(((u128)n + __umul64hi(n, v)) >> 1);
  u128 rem = ((u128)n << 63) - (u128)q * d;  // >= 0: q is not above the quotient
#pragma unroll 1
  for (int i = 0; i < 8 && rem >= (u128)d; ++i) {
    q += 1;
    rem -= d;
  }
  return q;
}

// ln(M * 2^E) for integer 1 <= M < 2^53.
__device__ __forceinline__ double fx_ln(uint64_t M, int E) {
  int q = 63 - __clzll(M);
  if ((u128)M * M >= ((u128)1 << (2 * q + 1))) q += 1;
  const int K = E + q;
  const uint64_t P = 1ull << q;
  const uint64_t n = M >= P ? M - P : P - M;
  const uint64_t d = M + P;
  if (n == 0) {
    if (K == 0) return 0.0;
    const u128 A = (u128)(uint64_t)(K > 0 ? K : -K) * 0xB17217F7D1CF79ACull;
    const double r = round_to_f64(A, -64);
    return K > 0 ? r : -r;
  }
  const int a = __clzll(n), b = __clzll(d);
  const uint64_t Q = quot_q63(n << a, d << b);  // |s| = Q 2^(b - a - 63)
  const int sh = a - b - 1;                     // >= 1
  const uint64_t s64 = sh >= 64 ? 0ull : (Q >> sh);
  const uint64_t z = __umul64hi(s64, s64);
  // sum_{i=1..12} z^i/(2i+1) in Q64; constants are floor(2^64 / (2i+1))
  uint64_t R = 0xFFFFFFFFFFFFFFFFull / 25u;
  R = 0xFFFFFFFFFFFFFFFFull / 23u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 21u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 19u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 17u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 15u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 13u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 11u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 9u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 7u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 5u + __umul64hi(z, R);
  R = 0xFFFFFFFFFFFFFFFFull / 3u + __umul64hi(z, R);
  const uint64_t F = __umul64hi(z, R);
  const u128 Lm = (u128)Q + __umul64hi(Q, F);  // |ln m| = Lm 2^(b - a - 62)
  const bool pos = M > P;                      // sign of ln m
  if (K == 0) {
    const double r = round_to_f64(Lm, b - a - 62);
    return pos ? r : -r;
  }
  const int rs = a - b - 2;  // |ln m| in Q64 = Lm >> rs
  const u128 LQ = rs >= 128 ? (u128)0 : (Lm >> rs);
  const u128 A = (u128)(uint64_t)(K > 0 ? K : -K) * 0xB17217F7D1CF79ACull;
  if (K > 0) return round_to_f64(pos ? A + LQ : A - LQ, -64);
  return -round_to_f64(pos ? A - LQ : A + LQ, -64);
}

// ln(x) of a positive finite binary64.
__device__ __forceinline__ double rt_ln(double x) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const int ef = (int)((bits >> 52) & 0x7FF);
  const uint64_t frac = bits & 0x000FFFFFFFFFFFFFull;
  return ef == 0 ? fx_ln(frac, -1074) : fx_ln(frac | (1ull << 52), ef - 1075);
}

// The odd integer x with u = x 2^-53 for 64 random bits.
__device__ __forceinline__ uint64_t bits_to_x(uint64_t bits) { return ((bits >> 12) << 1) | 1ull; }

// Exp(1) increment ln(1/u) (Eq. 24).
__device__ __forceinline__ double exp1_from_bits(uint64_t bits) { return -fx_ln(bits_to_x(bits), -53); }

__device__ __forceinline__ double exp1_draw(uint64_t seed, uint64_t g, uint32_t k, uint32_t n, uint32_t stream) {
  return exp1_from_bits(draw_bits(seed, g, k, n, stream));
}

}  // namespace rt

// Conversions between the library's Q1.63 fixed-point values (value x
// stored as the integer x 2^63) and FP32/FP64, with integer instructions
// only.  GB300 executes FP64 arithmetic, including conversions from and to
// 64-bit integers, at a small fraction of its FP32 rate: a streaming kernel
// doing three such operations per cell (e.g. rf = (float)((double)r * alpha
// / 2^63)) was bound by them, at about 0.4 of the copy bandwidth.  The
// rounding conversions round to nearest, ties to even, like cvt.rn.
#pragma once

#include <cstdint>

namespace ppr {

typedef unsigned long long u64;

// the float nearest to u * 2^E2 (u != 0 must land in the normal range)
template <int E2>
__device__ __forceinline__ float u64_to_f32(u64 u) {
  if (u == 0) return 0.f;
  const int lz = __clzll(u);
  const u64 m = u << lz;                        // leading one at bit 63
  uint32_t top = (uint32_t)(m >> 40);           // 24 significant bits
  const u64 rest = m & 0xFFFFFFFFFFull, half = 0x8000000000ull;
  top += (rest > half || (rest == half && (top & 1u))) ? 1u : 0u;
  // top's leading bit adds one to the exponent field; a carry out of the
  // 24 bits adds one more and leaves the fraction zero
  return __uint_as_float(((uint32_t)(63 - lz + E2 + 126) << 23) + top);
}

// the double nearest to u * 2^E2
template <int E2>
__device__ __forceinline__ double u64_to_f64(u64 u) {
  if (u == 0) return 0.0;
  const int lz = __clzll(u);
  const u64 m = u << lz;
  u64 top = m >> 11;                            // 53 significant bits
  const u64 rest = m & 0x7FFull, half = 0x400ull;
  top += (rest > half || (rest == half && (top & 1ull))) ? 1ull : 0ull;
  return __longlong_as_double((long long)(((u64)(63 - lz + E2 + 1022) << 52) + top));
}

// the float nearest to d * 2^-63 (a signed Q1.63 difference)
__device__ __forceinline__ float sfix_to_f32(long long d) {
  const float f = u64_to_f32<-63>(d < 0 ? 0ull - (u64)d : (u64)d);
  return d < 0 ? -f : f;
}

// the integer nearest to e * 2^63 (e in Q1.63 units), for |e| < 1; larger
// magnitudes, infinities and NaN give +-(2^63 - 1)
__device__ __forceinline__ long long f32_to_sfix(float e) {
  const uint32_t b = __float_as_uint(e);
  const int ex = (int)((b >> 23) & 0xFFu);
  if (ex == 0) return 0;                        // zero or subnormal: below 2^-63
  const u64 m = (u64)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 87;                       // |e| 2^63 = m 2^(ex - 150 + 63)
  u64 q;
  if (sh >= 40) {
    q = 0x7FFFFFFFFFFFFFFFull;
  } else if (sh >= 0) {
    q = m << sh;
  } else if (sh < -25) {
    q = 0;
  } else {
    const int k = -sh;
    q = m >> k;
    const u64 r = m & ((1ull << k) - 1ull), half = 1ull << (k - 1);
    q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
  }
  return (b >> 31) ? -(long long)q : (long long)q;
}

// floor(x * 2^63) for 0 <= x < 2 (truncation, as a float -> unsigned
// conversion); x <= 0 and NaN give 0, larger x 2^64 - 1
__device__ __forceinline__ u64 f32_to_ufix_trunc(float x) {
  const uint32_t b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xFFu);
  if ((b >> 31) || ex == 0) return 0;           // negative, zero, subnormal (below 2^-63)
  if (ex == 255 && (b & 0x7FFFFFu)) return 0;   // NaN
  const u64 m = (u64)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = ex - 87;                       // x 2^63 = m 2^(ex - 87)
  if (sh > 40) return ~0ull;
  if (sh >= 0) return m << sh;
  return sh <= -24 ? 0ull : m >> -sh;
}

// floor(mu * x) for mu < 2^63 and 0 <= x <= 1, exact (the 88-bit product
// mu * significand shifted down); negative x and NaN give 0
__device__ __forceinline__ u64 mul_fix_f32(u64 mu, float x) {
  const uint32_t b = __float_as_uint(x);
  const int ex = (int)((b >> 23) & 0xFFu);
  if ((b >> 31) || ex == 0 || ex == 255) return 0;
  const u64 m = (u64)((b & 0x7FFFFFu) | 0x800000u);
  const int s = 150 - ex;                       // x = m 2^-s
  if (s <= 0) return ~0ull;                     // x >= 2^23: outside the domain
  const u64 hi = __umul64hi(mu, m), lo = mu * m;
  if (s >= 128) return 0;
  if (s >= 64) return hi >> (s - 64);
  return (lo >> s) | (hi << (64 - s));
}

}  // namespace ppr

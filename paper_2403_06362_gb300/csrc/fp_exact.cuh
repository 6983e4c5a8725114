// fp_exact.cuh -- fp64 results computed on the integer pipes, bit for bit
// equal to the fp64 operations they replace.
//
// This GPU retires two fp64 lanes per clock per SM against 128 integer
// lanes, and its fp64 unit spends the same time on a warp instruction
// whatever the number of live lanes.  The fp64 transport kernels are bound by
// that unit, so every fp64 step whose exact result can be assembled from
// integer operations is moved off it:
//   two_u_minus_1  2u - 1 for a draw u = n 2^-53 (exact: (2n - 2^53) 2^-53)
//   floor_nonneg   floor(t) for 0 <= t < 2^63
//   abs_le         |x| <= h for h >= 0
//   recip_rn       1/y correctly rounded (IEEE round to nearest even)
//   llrint_nonneg  llrint(v) for 0 <= v < 2^62
//   okey, d_lt ..  comparisons of doubles (sign-magnitude order keys)
//   mul_small      RN(j h) for a small integer j
// All of them compile for host and device; the host copies let tests compare
// them with the host's IEEE arithmetic.
#pragma once
#include <cstdint>

#include "mc_log.cuh"  // to_bits, from_bits

namespace mcx {

using mclog::from_bits;
using mclog::to_bits;

__host__ __device__ __forceinline__ int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ float rcp_f32(float x) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}

// 2u - 1 for u = n 2^-53, 0 <= n < 2^53: the double (2n - 2^53) 2^-53,
// exact (|2n - 2^53| <= 2^53), +0 for n = 2^52.
__host__ __device__ __forceinline__ double two_u_minus_1(uint64_t n) {
  const long long w = (long long)(n << 1) - (1ll << 53);
  if (w == 0) return 0.0;
  const uint64_t sign = w < 0 ? (1ull << 63) : 0ull;
  const uint64_t a = w < 0 ? (uint64_t)(-w) : (uint64_t)w;  // 2 .. 2^53
  if (a == (1ull << 53)) return -1.0;
  const int lz = clz64(a);  // 11 .. 62
  // leading 1 moved to bit 52; it carries into the exponent field, so the
  // word to add is (biased exponent - 1) << 52 with biased = 1033 - lz
  return from_bits(sign | ((a << (lz - 11)) + ((uint64_t)(1032 - lz) << 52)));
}

// floor(t) for 0 <= t < 2^63 (t finite, not negative zero excluded).
__host__ __device__ __forceinline__ uint64_t floor_nonneg(double t) {
  const uint64_t b = to_bits(t);
  const int e = (int)(b >> 52) - 1023;
  if (e < 0) return 0ull;
  const uint64_t m = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
  return e <= 52 ? m >> (52 - e) : m << (e - 52);
}

// |x| <= h for h >= 0 (finite): non-negative doubles order like their bits.
__host__ __device__ __forceinline__ bool abs_le(double x, double h) {
  return (to_bits(x) & ~(1ull << 63)) <= to_bits(h);
}

// q = RN(2^105 / M) for 2^52 < M < 2^53 (ties cannot occur: 2^106 = (2q + 1) M
// would make M a power of two).  With m = M 2^-52 = F (1 + r), F = 1 + j/1024
// the left end of m's cell (the table of 2^63 / F that the logarithm uses)
// and 0 <= r < 2^-10,
//   2^53 / m = (2^53 / F) (1 - r (1 - r (1 - r (1 - r (1 - r))))) + O(r^6 < 2^-60)
// by Horner's rule on non-negative fixed point (the inner terms on 32 bits)
// puts q within a unit; an exact remainder fixes it and rounds.
__host__ __device__ __forceinline__ uint64_t recip_mantissa(uint64_t M) {
  const int j = (int)((M >> 42) & 1023ull);
#ifdef __CUDA_ARCH__
  const uint64_t inv = __ldg(&mclog::dev::kInvF[j]);  // 2^63 / F
#else
  const uint64_t inv = mclog::host::kInvF[j];
#endif
  const uint64_t R = mclog::umulhi_((M & ((1ull << 42) - 1ull)) << 22, inv);  // r 2^73
  const uint32_t r32 = (uint32_t)(R >> 31);                                     // r 2^42
  uint32_t t = (1u << 31) - (r32 >> 11);                       // T3 = 1 - r, scale 2^31
  t = (1u << 31) - (mclog::umulhi32_(r32, t) >> 10);           // T2 = 1 - r T3, scale 2^31
  t = (1u << 31) - mclog::umulhi32_(r32, t);                   // T1 - (1 - 2^-10), scale 2^41
  const uint64_t rt = ((uint64_t)(uint32_t)(R >> 32) * t + (((uint64_t)(uint32_t)R * t) >> 32)) >> 19;
  const uint64_t t0 = (1ull << 63) - ((R >> 10) - (R >> 20)) - rt;         // T0 = 1 - r T1, scale 2^63
  const uint64_t S = (1ull << 63) - (mclog::umulhi_(R, t0) >> 9);          // 1 / (1 + r), scale 2^63
  uint64_t q = mclog::umulhi_(inv, S) >> 9;                                // ~ 2^53 / m
  // exact remainder r = 2^105 - q M (|r| < 2^63: the low words decide), then round
  long long rem = (long long)(0ull - q * M);
  for (int i = 0; i < 4 && rem < 0; ++i) { --q; rem += (long long)M; }
  for (int i = 0; i < 4 && rem >= (long long)M; ++i) { ++q; rem -= (long long)M; }
  if ((uint64_t)rem * 2ull > M) ++q;
  return q;
}

// RN(1 / y) on the integer pipes for normal y whose reciprocal is normal
// (biased exponent 1..2044); the library division otherwise (zero,
// subnormal, huge, inf, NaN).
__host__ __device__ __forceinline__ double recip_rn(double y) {
  const uint64_t b = to_bits(y);
  const uint64_t sign = b & (1ull << 63);
  const uint32_t E = (uint32_t)(b >> 52) & 0x7FFu;
  if (E == 0u || E > 2044u) return 1.0 / y;
  const uint64_t frac = b & ((1ull << 52) - 1ull);
  if (frac == 0ull) return from_bits(sign | ((uint64_t)(2046u - E) << 52));  // a power of two
  const uint64_t q = recip_mantissa(frac | (1ull << 52));  // in [2^52, 2^53)
  return from_bits(sign | (((uint64_t)(2045u - E) << 52) + (q - (1ull << 52))));
}

// llrint(v) (round half to even) for 0 <= v < 2^62, from the bits.
__host__ __device__ __forceinline__ long long llrint_nonneg(double v) {
  const uint64_t b = to_bits(v);
  const int e = (int)(b >> 52) - 1023;
  if (e < -1) return 0;  // v < 1/2
  const uint64_t m = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
  if (e >= 52) return (long long)(m << (e - 52));
  const int sh = 52 - e;  // 1..53
  const uint64_t q = m >> sh, rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  return (long long)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
}

// Order key of a non-NaN double: a < b  <=>  okey(a) < okey(b); -0 and +0
// share the key 0.
__host__ __device__ __forceinline__ long long okey(double x) {
  const uint64_t b = to_bits(x);
  const long long m = (long long)(b & ~(1ull << 63));
  return (b >> 63) ? -m : m;
}
__host__ __device__ __forceinline__ bool d_lt(double a, double b) { return okey(a) < okey(b); }
__host__ __device__ __forceinline__ bool d_pos(double a) { return (long long)to_bits(a) > 0; }        // a > 0
__host__ __device__ __forceinline__ bool d_neg(double a) { return to_bits(a) > (1ull << 63); }         // a < 0
__host__ __device__ __forceinline__ bool d_zero(double a) { return (to_bits(a) << 1) == 0ull; }        // a == 0

// RN(j h) for an integer 0 <= j < 2^11 and a normal h > 0 whose product
// stays normal: the exact product m_h j has at most 64 bits, rounded once.
__host__ __device__ __forceinline__ double mul_small(uint32_t j, double h) {
  if (j == 0u) return 0.0;
  const uint64_t b = to_bits(h);
  const uint64_t m = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
  const uint64_t p = m * (uint64_t)j;  // < 2^64
  const int lz = clz64(p);             // 0..11
  const int sh = 11 - lz;              // bits below the 53 kept
  uint64_t q = p >> sh;
  if (sh > 0) {
    const uint64_t rem = p & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;  // may carry to 2^53
  }
  // value = q 2^(E_h + sh - 1075): biased exponent E_h + sh with q's leading
  // 1 at bit 52 (a carry to 2^53 moves into the exponent by itself)
  return from_bits((b & ~((1ull << 52) - 1ull)) + ((uint64_t)sh << 52) + (q - (1ull << 52)));
}

// A positive normal x as q 2^-s with a 32-bit q in [2^31, 2^32) (truncated),
// and floor(a x) within one for 0 <= a from it: a lookup guess that an exact
// comparison then corrects.
__host__ __device__ __forceinline__ void fixed_of(double x, uint32_t& q, int& s) {
  const uint64_t b = to_bits(x);
  q = (uint32_t)((((b & ((1ull << 52) - 1ull)) | (1ull << 52))) >> 21);
  s = 31 - ((int)(b >> 52) - 1023);
}
__host__ __device__ __forceinline__ uint64_t guess_floor_mul(double a, uint32_t q, int s) {
  const uint64_t b = to_bits(a);
  if ((b << 1) == 0ull) return 0ull;
  const int e = (int)(b >> 52) - 1023;
  const uint64_t m32 = (((b & ((1ull << 52) - 1ull)) | (1ull << 52))) >> 21;  // a ~ m32 2^(e - 31)
  const int sh = 31 + s - e;
  if (sh >= 64) return 0ull;
  if (sh <= 0) return 1ull << 40;
  return (m32 * (uint64_t)q) >> sh;
}

// llrint(w 2^32) for w >= 0 (2^32 w < 2^62): the scaling as an exponent add.
__host__ __device__ __forceinline__ long long fix32_nonneg(double w) {
  const uint64_t b = to_bits(w);
  if ((b >> 52) == 0ull) return 0;  // zero or below 2^-1022
  return llrint_nonneg(from_bits(b + (32ull << 52)));
}

// x 2^k for a normal x whose product stays normal (an exponent add).
__host__ __device__ __forceinline__ double scale_pow2(double x, int k) {
  return from_bits(to_bits(x) + ((uint64_t)(int64_t)k << 52));
}

}  // namespace mcx

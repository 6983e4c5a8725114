// mc_log.cuh -- ln(1 - u) for a uniform u = n 2^-53 in [0, 1): the logarithm
// of the fp64 flight distance d = -ln(1 - u) / Sigma_t, computed on the
// integer pipes.
//
// This GPU retires two fp64 lanes per clock per SM against 128 integer
// lanes, so the logarithm is evaluated in fixed point with integer
// operations and rounded once to the nearest double.  Method: the table
// reduction of P. T. P. Tang, "Table-driven implementation of the logarithm
// function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990.  With
// x = 1 - u = K 2^-53 (K = 2^53 - n, exact) = 2^e m, m in [1, 2), and
// F = 1 + (2j+1)/256 the midpoint of m's cell among 128 equal cells,
//   ln x = e ln 2 + ln F + ln(1 + r),  r = (m - F) / F,  |r| < 2^-8,
// where m - F is an exact integer difference, r is formed with a 64-bit
// reciprocal of F (scale 2^71), ln(1 + r) comes from its series through r^8
// by Horner's rule on 64-bit signed fixed point (scale 2^62; the terms from
// r^5 on, below 2^-42, on 32 bits), and the sum is
// accumulated on 128 bits with scale 2^90 (ln 2 and ln F from 128-bit
// tables).  For u < 2^-8 (x so close to 1 that e ln 2 + ln F would cancel)
// -ln(1 - u) = u (1 + u/2 + ... + u^8/9) is used instead, relative to u.
// The absolute error before the final rounding is below 2^-66 while the
// result is at least 2^-8 in magnitude (relatively below 2^-60 in the
// small-u branch), so the result is the correctly rounded logarithm except
// within a few hundredths of an ulp of a rounding tie.  The code is plain
// integer arithmetic, identical on host and device; tests compare it with a
// 40-digit decimal logarithm and with the host C library.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

namespace mclog {

#define MC_LOG_CONST static constexpr
#define MC_LOG_TABLE static __device__ const
#define MC_LOG_COEF static __constant__ const
namespace dev {
#include "log_table.inc"
}
#undef MC_LOG_TABLE
#undef MC_LOG_COEF
#define MC_LOG_TABLE static const
#define MC_LOG_COEF static const
namespace host {
#include "log_table.inc"
}
#undef MC_LOG_TABLE
#undef MC_LOG_COEF
#undef MC_LOG_CONST

__host__ __device__ __forceinline__ uint64_t to_bits(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  std::memcpy(&b, &v, sizeof b);
  return b;
#endif
}

__host__ __device__ __forceinline__ double from_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, sizeof v);
  return v;
#endif
}

__host__ __device__ __forceinline__ int clz64_(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ uint64_t umulhi_(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ long long smulhi_(long long a, long long b) {
#ifdef __CUDA_ARCH__
  return __mul64hi(a, b);
#else
  return (long long)(((__int128)a * b) >> 64);
#endif
}

// A 128-bit two's-complement integer.
struct W128 {
  uint64_t lo, hi;
};

__host__ __device__ __forceinline__ W128 add128(W128 a, W128 b) {
  W128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}

__host__ __device__ __forceinline__ W128 sub128(W128 a, W128 b) {
  W128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}

__host__ __device__ __forceinline__ int mulhi32_(int a, int b) {
#ifdef __CUDA_ARCH__
  return __mulhi(a, b);
#else
  return (int)(((long long)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ W128 neg128(W128 a) {
  W128 r;
  r.lo = 0ull - a.lo;
  r.hi = ~a.hi + (a.lo == 0ull ? 1ull : 0ull);
  return r;
}

// a 2^-scale as the nearest double (round half to even), a > 0, the result
// normal.
__host__ __device__ __forceinline__ double w128_to_double(W128 a, int scale) {
  const int lz = a.hi ? clz64_(a.hi) : 64 + clz64_(a.lo);
  const int top = 127 - lz;  // position of the leading 1
  uint64_t m64;              // the leading 64 bits, leading 1 at bit 63
  bool sticky;
  if (top >= 63) {
    const int sh = top - 63;  // 0..64
    if (sh == 0) {
      m64 = a.lo;
      sticky = false;
    } else if (sh < 64) {
      m64 = (a.hi << (64 - sh)) | (a.lo >> sh);
      sticky = (a.lo << (64 - sh)) != 0ull;
    } else {
      m64 = a.hi;
      sticky = a.lo != 0ull;
    }
  } else {
    m64 = a.lo << (63 - top);
    sticky = false;
  }
  uint64_t m53 = m64 >> 11;
  const uint64_t rest = m64 & 0x7FFull;
  if (rest > 0x400ull || (rest == 0x400ull && (sticky || (m53 & 1ull)))) ++m53;  // may carry to 2^53
  const uint64_t biased = (uint64_t)(top - scale + 1023);
  return from_bits(((biased - 1ull) << 52) + m53);  // the leading 1 adds one to the exponent
}

// The same for 2^82 <= a < 2^96 (the leading 1 at bit 82..95 of the high
// word's range), without branches.
__host__ __device__ __forceinline__ double w128_to_double_hi(W128 a, int scale) {
  const int top = 127 - clz64_(a.hi);  // 82..95
  const int sh = top - 63;             // 19..32
  const uint64_t m64 = (a.hi << (64 - sh)) | (a.lo >> sh);
  const bool sticky = (a.lo << (64 - sh)) != 0ull;
  uint64_t m53 = m64 >> 11;
  const uint64_t rest = m64 & 0x7FFull;
  if (rest > 0x400ull || (rest == 0x400ull && (sticky || (m53 & 1ull)))) ++m53;
  return from_bits(((uint64_t)(top - scale + 1022) << 52) + m53);
}

// ln(1 - u) for u = n 2^-53, 0 <= n < 2^53: a double <= 0 (+0 for n = 0).
__host__ __device__ __forceinline__ double log1m_n(uint64_t n) {
#ifdef __CUDA_ARCH__
  using namespace dev;
#define MC_LOG_LD(a, i) __ldg(&(a)[(i)])
#else
  using namespace host;
#define MC_LOG_LD(a, i) (a)[(i)]
#endif
  if (n < (1ull << 45)) {  // u < 2^-8: -u (1 + u/2 + ... + u^8/9)
    if (n == 0ull) return 0.0;
    const long long U = (long long)(n << 18);  // u 2^71
    long long t = kLn1mB[8];
#pragma unroll
    for (int k = 7; k >= 0; --k) t = kLn1mB[k] + (smulhi_(U, t) >> 7);  // scale 2^62
    W128 p;
    p.lo = n * (uint64_t)t;
    p.hi = umulhi_(n, (uint64_t)t);  // n t = -ln(1 - u) 2^115
    return -w128_to_double(p, 115);
  }
  const uint64_t K = (1ull << 53) - n;  // x = K 2^-53, 1 <= K < 2^53 - 2^45
  const int lz = clz64_(K);             // 12..63
  const int e = 10 - lz;                // x = 2^e m
  const uint64_t mant = K << (lz - 11);  // m 2^52, leading 1 at bit 52
  const int j = (int)((mant >> 45) & 127ull);
  const long long D = (long long)mant - (long long)((1ull << 52) + ((uint64_t)(2 * j + 1) << 44));  // (m - F) 2^52
  const uint64_t inv = MC_LOG_LD(kInvF, j);                                                        // 2^64 / F
  const uint64_t ad = D < 0 ? (uint64_t)(-D) : (uint64_t)D;
  const uint64_t pr = (umulhi_(ad, inv) << 19) | ((ad * inv) >> 45);  // |r| 2^71
  const long long R = D < 0 ? -(long long)pr : (long long)pr;
  // ln(1 + r) = r (1 + r (c2 + r (c3 + r (c4 + r Q)))), Q = c5 + r (c6 + r (c7 + r c8)):
  // |r^5 Q| < 2^-42, so Q needs only 32-bit arithmetic (scale 2^30, r at 2^39)
  const int R32 = (int)(R >> 32);
  int q = (int)(kLn1pC[7] >> 32);
  q = (int)(kLn1pC[6] >> 32) + (mulhi32_(R32, q) >> 7);
  q = (int)(kLn1pC[5] >> 32) + (mulhi32_(R32, q) >> 7);
  q = (int)(kLn1pC[4] >> 32) + (mulhi32_(R32, q) >> 7);
  long long t = (long long)q << 32;  // scale 2^62
#pragma unroll
  for (int k = 3; k >= 0; --k) t = kLn1pC[k] + (smulhi_(R, t) >> 7);
  // ln(1 + r) 2^71 = (R t) >> 62, then to scale 2^90 (sign-extended)
  const long long ph = smulhi_(R, t);
  const uint64_t pl = (uint64_t)R * (uint64_t)t;
  const long long p71 = (long long)(((uint64_t)ph << 2) | (pl >> 62));
  W128 p;
  p.lo = (uint64_t)p71 << 19;
  p.hi = (uint64_t)(p71 >> 45);
  // -ln x = |e| ln 2 - ln F - ln(1 + r) > 2^-8, on 128 bits with scale 2^90
  const uint64_t ae = (uint64_t)(-e);
  W128 a;
  a.lo = ae * kLn2Lo;
  a.hi = umulhi_(ae, kLn2Lo) + ae * kLn2Hi;
  W128 f;
  f.lo = MC_LOG_LD(kLnFLo, j);
  f.hi = MC_LOG_LD(kLnFHi, j);
  a = sub128(sub128(a, f), p);
#undef MC_LOG_LD
  return -w128_to_double_hi(a, 90);
}

// ln(1 - u) for a double u = n 2^-53 in [0, 1) (every uniform of the library).
__host__ __device__ __forceinline__ double log1m(double u) {
  const uint64_t b = to_bits(u);
  if (b == 0ull) return 0.0;
  const int e = (int)(b >> 52) - 1023;  // u = (1.f) 2^e, e in [-53, -1]
  const uint64_t m = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
  return log1m_n(m >> (-e - 1));  // n = u 2^53 = m 2^(e + 1)
}

}  // namespace mclog

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
// F = 1 + j/1024 the left end of m's cell among 1024 equal cells,
//   ln x = e ln 2 + ln F + ln(1 + r),  r = (m - F) / F,  0 <= r < 2^-10,
// where m - F is the exact low 42 bits of m's mantissa, r is formed with a
// 64-bit reciprocal of F (scale 2^73), ln(1 + r) comes from its series
// through r^6 by Horner's rule on non-negative fixed point (the inner terms
// on 32 bits, the outer two on 64), and the sum is
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

__host__ __device__ __forceinline__ uint32_t umulhi32_(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
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

// The same for 2^82 <= a < 2^96, on the three low 32-bit words (the high
// word is below 2^32), without branches.
__host__ __device__ __forceinline__ uint32_t clz32_(uint32_t x) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__clz((int)x);
#else
  return x ? (uint32_t)__builtin_clz(x) : 32u;
#endif
}
// The low word of (hi:lo) >> s, 0 <= s <= 32.
__host__ __device__ __forceinline__ uint32_t fsr32_(uint32_t lo, uint32_t hi, uint32_t s) {
#ifdef __CUDA_ARCH__
  return __funnelshift_rc(lo, hi, s);
#else
  return (uint32_t)((((uint64_t)hi << 32) | lo) >> s);
#endif
}
__host__ __device__ __forceinline__ double w128_to_double_hi(W128 a, int scale) {
  const uint32_t h = (uint32_t)a.hi, l1 = (uint32_t)(a.lo >> 32), l0 = (uint32_t)a.lo;
  const int top = 95 - (int)clz32_(h);  // 82..95
  const uint32_t sh = (uint32_t)(top - 63);  // 19..32
  const uint64_t m64 = ((uint64_t)fsr32_(l1, h, sh) << 32) | fsr32_(l0, l1, sh);  // bits sh..sh+63
  const bool sticky = (l0 << (32u - sh)) != 0u;  // any of the bits below sh
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
  const int j = (int)((mant >> 42) & (uint64_t)(kLogCells - 1));  // m in [F_j, F_j + 2^-10)
  const uint64_t D = mant & ((1ull << 42) - 1ull);                // (m - F_j) 2^52, exact
  const uint64_t R = umulhi_(D << 22, MC_LOG_LD(kInvF, j));       // r 2^73 (2^63 / F_j in the table)
  // ln(1 + r) = r P, P = 1 - r Q0, Q0 = 1/2 - r Q1, Q1 = 1/3 - r Q2, Q2 = 1/4 - r Q3,
  // Q3 = 1/5 - r/6 (the r^7 term is below 2^-72): r and Q3, Q2 and Q1 - 85/256
  // on 32 bits, Q0 and P on 64 (scale 2^63); every quantity is non-negative.
  const uint32_t r32 = (uint32_t)(R >> 31);                        // r 2^42
  uint32_t q = kQ3 - (umulhi32_(r32, kQ4) >> 10);                  // Q3 2^32
  q = (1u << 30) - (umulhi32_(r32, q) >> 10);                      // Q2 2^32
  q = kQ1B - (umulhi32_(r32, q) >> 1);                             // (Q1 - 85/256) 2^41
  const uint64_t rq = ((uint64_t)(uint32_t)(R >> 32) * q + (((uint64_t)(uint32_t)R * q) >> 32)) >> 19;
  const uint64_t q0 = (1ull << 62) - (((R >> 10) * 85ull) >> 8) - rq;  // Q0 2^63
  const uint64_t P = (1ull << 63) - (umulhi_(R, q0) >> 9);            // P 2^63
  const uint64_t p72 = umulhi_(R, P);                                 // ln(1 + r) 2^72
  W128 p;
  p.lo = p72 << 18;
  p.hi = p72 >> 46;
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

// mc_log.cuh -- ln(1 - u) for a uniform u in [0, 1): the logarithm of the
// fp64 flight distance d = -ln(1 - u) / Sigma_t.
//
// Method: table-driven logarithm after P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990.  With x = 1 - u = 2^k m, m in [1, 2), and
// F = 1 + (2j+1)/256 the midpoint of m's cell among 128 equal cells,
//   ln x = k ln 2 + ln F + ln(1 + r),  r = (m - F) / F,  |r| < 2^-9,
// where k ln2_hi + ln(F)_hi is exact (both parts are multiples of 2^-42) and
// ln(1 + r) comes from its Taylor series through r^6.  For u < 2^-8, where x
// is so close to 1 that k ln 2 + ln F would cancel, the Taylor series of
// ln(1 - u) through u^8 is used instead.  The table path costs 14 fp64
// operations (the library logarithm costs about 30 on this GPU, whose fp64
// unit is narrow) and stays within about one ulp of the correctly rounded
// value; tests compare it with the host C library.  The code is the same on
// host and device (explicit fma, no contraction), so both give the same bits.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

namespace mclog {

#define MC_LOG_CONST static constexpr
#define MC_LOG_TABLE static __device__ const
namespace dev {
#include "log_table.inc"
}
#undef MC_LOG_TABLE
#define MC_LOG_TABLE static const
namespace host {
#include "log_table.inc"
}
#undef MC_LOG_TABLE
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

// ln(1 - u) for 0 <= u < 1 with 1 - u exact (u a multiple of 2^-53, as every
// uniform of the library is).
__host__ __device__ __forceinline__ double log1m(double u) {
  if (to_bits(u) < to_bits(0x1p-8)) {  // u < 2^-8 (u >= 0): -(u + u^2 q), q = 1/2 + u/3 + ... + u^6/8
    double q = 1.0 / 8.0;
    q = fma(q, u, 1.0 / 7.0);
    q = fma(q, u, 1.0 / 6.0);
    q = fma(q, u, 1.0 / 5.0);
    q = fma(q, u, 1.0 / 4.0);
    q = fma(q, u, 1.0 / 3.0);
    q = fma(q, u, 1.0 / 2.0);
    return 0.0 - fma(u, u * q, u);  // u^2 q < u 2^-9: one rounding of the sum dominates; +0 at u = 0
  }
#ifdef __CUDA_ARCH__
  using namespace dev;
#define MC_LOG_LD(a, i) __ldg(&(a)[(i)])
#else
  using namespace host;
#define MC_LOG_LD(a, i) (a)[(i)]
#endif
  const double x = 1.0 - u;  // exact, in [2^-53, 1 - 2^-8]
  const uint64_t bits = to_bits(x);
  const int k = (int)(bits >> 52) - 1023;
  const uint64_t mant = bits & ((1ull << 52) - 1ull);
  const int j = (int)(mant >> 45);
  const double m = from_bits(0x3FF0000000000000ull | mant);
  const double F = from_bits(0x3FF0000000000000ull | ((uint64_t)(2 * j + 1) << 44));
  const double r = (m - F) * MC_LOG_LD(kInvF, j);  // m - F exact (Sterbenz)
  double q = -1.0 / 6.0;
  q = fma(q, r, 1.0 / 5.0);
  q = fma(q, r, -1.0 / 4.0);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -1.0 / 2.0);
  const double p = fma(r * r, q, r);  // ln(1 + r)
  const double kd = (double)k;
  const double s = fma(kd, kLn2Hi, MC_LOG_LD(kLnFHi, j));  // exact
  const double t = fma(kd, kLn2Lo, MC_LOG_LD(kLnFLo, j)) + p;
#undef MC_LOG_LD
  return s + t;
}

}  // namespace mclog

// mc_device.cuh -- device-side LCG, skip-ahead, hash and uniform conversion.
//
// Everything here is integer arithmetic that the GB300 SM runs on its
// integer pipes: a 64-bit product is one IMAD.WIDE.U32 plus two IMADs, and
// the fp64 uniform is assembled from integer pieces (clz, funnel shift,
// exponent add) so that no fp64 instruction is issued on the draw path
// (fp64 is a narrow unit on this part).
#pragma once
#include <cstdint>

namespace mcd {

// Listing 1 multiplier of the modified murmur_hash64a.
constexpr uint64_t kMurmurM = 0xC6A4A7935BD1E995ull;

// Parameters of Eq. (1) as the kernels use them.  The recurrence runs mod
// 2^64 in registers; reduction mod 2^m is a ring homomorphism from Z/2^64,
// so the low m bits of the 64-bit state are the m-bit state, and the mask
// is applied only where a state leaves the kernel.
struct Lcg {
  uint64_t g, c, mask;
  uint32_t m;
};

__host__ __device__ __forceinline__ uint64_t mask_of(uint32_t m) {
  return m >= 64 ? ~0ull : ((1ull << m) - 1ull);
}

__device__ __forceinline__ uint64_t lcg_step(uint64_t x, uint64_t g, uint64_t c) {
  return g * x + c;  // wraps mod 2^64
}

// Affine map x -> a*x + b (mod 2^64): the map of some number of LCG steps.
struct Affine {
  uint64_t a, b;
};

__host__ __device__ __forceinline__ Affine compose(Affine outer, Affine inner) {
  // outer(inner(x)) = oa*(ia*x + ib) + ob
  return Affine{outer.a * inner.a, outer.a * inner.b + outer.b};
}

__host__ __device__ __forceinline__ uint64_t apply(Affine f, uint64_t x) { return f.a * x + f.b; }

// Eq. (2), Brown's binary method: the map of k steps from the map of one
// step, by squaring (map of 2^(j+1) steps = map of 2^j steps applied twice)
// and composing the squares selected by the bits of k.
__host__ __device__ __forceinline__ Affine skip_map(uint64_t g, uint64_t c, uint64_t k) {
  Affine acc{1ull, 0ull};
  Affine sq{g, c};
  while (k) {
    if (k & 1ull) acc = compose(sq, acc);
    sq = compose(sq, sq);
    k >>= 1;
  }
  return acc;
}

// Section 4, Listing 1 and Eq. 3: one mixing step multiplies by the murmur
// constant (mod 2^64) and folds the product's top 17 bits into its low bits;
// the hash mixes the key, multiplies it by the constant again, combines it by
// XOR with the mixed seed (the seed first XORed with 8 times the constant)
// and mixes the result once more.
__host__ __device__ __forceinline__ uint64_t subhash(uint64_t x) {
  const uint64_t t = x * kMurmurM;
  return t ^ (t >> 47);
}

// The seed half of the hash, computed once per parent seed.
__host__ __device__ __forceinline__ uint64_t seed_hash_of(uint64_t s) {
  return subhash(s ^ (8ull * kMurmurM));
}

__host__ __device__ __forceinline__ uint64_t hash_with(uint64_t k, uint64_t seed_hash) {
  return subhash(seed_hash ^ (subhash(k) * kMurmurM));
}

__host__ __device__ __forceinline__ uint64_t hash64(uint64_t k, uint64_t s) {
  return hash_with(k, seed_hash_of(s));
}

// Exact conversion of an integer n < 2^53 to the double n * 2^-53, built
// from integer operations: normalise n so that its top bit sits at bit 52,
// then add the biased exponent one below the true one (the leading 1 at bit
// 52 carries into the exponent field).  For n in [2^52, 2^53) the value is
// in [0.5, 1) with biased exponent 1022 = 1033 - clz64(n); in general the
// word to add is (1032 - clz64(n)) << 52.
__device__ __forceinline__ double u53_to_double(uint32_t hi, uint32_t lo) {
  uint32_t rhi, rlo;
  if (hi != 0u) {  // all but 2^-21 of the draws
    const uint32_t lz = __clz(hi);  // 11..31 since hi < 2^21
    const uint32_t s = lz - 11u;
    rhi = __funnelshift_l(lo, hi, s) + ((1032u - lz) << 20);
    rlo = lo << s;
  } else if (lo != 0u) {
    const uint32_t lz = 32u + __clz(lo);  // 32..63
    const uint64_t nn = (uint64_t)lo << (lz - 11u);
    const uint64_t bits = nn + ((uint64_t)(1032u - lz) << 52);
    rhi = (uint32_t)(bits >> 32);
    rlo = (uint32_t)bits;
  } else {
    rhi = 0u;
    rlo = 0u;
  }
  return __hiloint2double((int)rhi, (int)rlo);
}

// Uniform of an (unmasked, mod 2^64) state for the common m = 63: bits
// 10..62 of x, i.e. the top 53 of the 63 state bits.
__device__ __forceinline__ double u01_m63(uint64_t x) {
  const uint32_t xlo = (uint32_t)x, xhi = (uint32_t)(x >> 32);
  const uint32_t lo = __funnelshift_r(xlo, xhi, 10);
  const uint32_t hi = (xhi << 1) >> 11;
  return u53_to_double(hi, lo);
}

// Pieces of the digest kernels' branch-free draw for m = 63.  They run on
// the doubled state z = 2x (mod 2^64), which follows z' = g z + 2c and
// holds the uniform's 53 bits n = z >> 11 at the top of the word.  With s
// the normalising shift of n (s = clz(z_hi) when z_hi != 0), the fp64 bit
// pattern of u = n 2^-53 is (1021 - s) 2^52 + (n << s): n << s has its
// leading 1 at bit 52, which carries one into the exponent field.

// clz(v) for v != 0; all ones for v = 0 (PTX bfind.shiftamt).
__device__ __forceinline__ uint32_t clz_or_ones(uint32_t v) {
  uint32_t r;
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(r) : "r"(v));
  return r;
}

// v << s with the shift clamped (PTX shl: 0 for s >= 32).
__device__ __forceinline__ uint32_t shl_clamped(uint32_t v, uint32_t s) {
  uint32_t r;
  asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(s));
  return r;
}

// n << s for s = clz_or_ones(z_hi) < 32 (exact then: n < 2^(53 - s)); any
// value for s = all ones.
__device__ __forceinline__ uint64_t n_shifted_m63(uint64_t z, uint32_t s) {
  const uint32_t zl = (uint32_t)z, zh = (uint32_t)(z >> 32);
  const uint32_t nl = __funnelshift_r(zl, zh, 11), nh = zh >> 11;
  return ((uint64_t)__funnelshift_l(nl, nh, s) << 32) | shl_clamped(nl, s);
}

// Adds s to a sum kept as the bit pattern of an fp32 subnormal (value
// s 2^-149), on the fp32 pipe.  The sum is exact while it stays below 2^24
// units; the all-ones s of a z_hi = 0 draw is a NaN pattern and turns the
// sum into a NaN, which marks the stream.  Explicit PTX, so that no
// flush-to-zero setting can apply.
__device__ __forceinline__ float add_count(float acc, uint32_t s) {
  float r;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(acc), "f"(__uint_as_float(s)));
  return r;
}

// True if a sum kept by add_count met a z_hi = 0 draw (its pattern is a NaN).
__device__ __forceinline__ bool count_marked(float acc) { return __float_as_uint(acc) > 0x7f800000u; }

// Uniform for any 1 <= m <= 64.
__device__ __forceinline__ double u01_any(uint64_t x, uint32_t m) {
  if (m >= 53u) {
    const uint64_t n = (x & mask_of(m)) >> (m - 53u);
    return u53_to_double((uint32_t)(n >> 32), (uint32_t)n);
  }
  // m < 53: x * 2^-m == (x << (53 - m)) * 2^-53, still below 2^53.
  const uint64_t n = (x & mask_of(m)) << (53u - m);
  return u53_to_double((uint32_t)(n >> 32), (uint32_t)n);
}

// The integer n of a draw's uniform u = n 2^-53 (0 <= n < 2^53): the top
// 53 of the m state bits (m >= 53), or the state shifted up (m < 53).
template <int M>
__device__ __forceinline__ uint64_t u53(uint64_t x, uint32_t m) {
  if constexpr (M == 63) {
    return (x << 1) >> 11;
  } else {
    return m >= 53u ? (x & mask_of(m)) >> (m - 53u) : (x & mask_of(m)) << (53u - m);
  }
}

template <int M>
__device__ __forceinline__ double u01(uint64_t x, uint32_t m) {
  if constexpr (M == 63) {
    return u01_m63(x);
  } else {
    return u01_any(x, m);
  }
}

__device__ __forceinline__ uint64_t dbits(double v) { return (uint64_t)__double_as_longlong(v); }

// Warp-level aggregation of per-lane counters before their global atomics:
// a run's counters for one problem share a cache line, so one atomic per lane
// and counter would all queue at the same L2 slice.  Called by a full,
// converged warp.
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
// Warp-aggregated int64 tally add.  The lanes that arrive here together
// (__activemask) and add to the same address form one group
// (__match_any_sync); the group's values are summed and its lowest lane
// issues the one atomic.  The sum runs on three 32-bit reductions of 26-,
// 26- and 12-bit pieces of each value: 32 pieces of at most 26 bits sum
// below 2^31, so every partial is exact and the recombined total equals
// the 64-bit sum mod 2^64, the same value the group's separate atomics
// would have added.  Integer addition is associative, so the tally bits do
// not depend on how the lanes happened to group.
__device__ __forceinline__ void warp_agg_add(unsigned long long* p, unsigned long long v) {
  const unsigned act = __activemask();
  const unsigned peers = __match_any_sync(act, reinterpret_cast<unsigned long long>(p));
  const unsigned lane = threadIdx.x & 31u;
  if (peers == (1u << lane)) {  // alone on this address: no reduction
    atomicAdd(p, v);
    return;
  }
  const unsigned s0 = __reduce_add_sync(peers, (unsigned)v & 0x3ffffffu);
  const unsigned s1 = __reduce_add_sync(peers, (unsigned)(v >> 26) & 0x3ffffffu);
  const unsigned s2 = __reduce_add_sync(peers, (unsigned)(v >> 52));
  if (lane == (unsigned)(__ffs(peers) - 1))
    atomicAdd(p, (unsigned long long)s0 + ((unsigned long long)s1 << 26) + ((unsigned long long)s2 << 52));
}

// The problem index all lanes with counts share: -1 when no lane has counts,
// -2 when lanes hold counts of different problems.
__device__ __forceinline__ int warp_common_prob(int prob) {
  const int p = __reduce_max_sync(0xffffffffu, prob);
  return __any_sync(0xffffffffu, prob >= 0 && prob != p) ? -2 : p;
}

}  // namespace mcd

// rng.cu -- seeding and draw kernels behind mc_seed_hash, mc_seed_stride
// and mc_lcg_draw.
//
// Seeding (Section 3, Eq. 2 and Section 4, Listing 1 / Eq. 3) is bound by
// the HBM store of 8 bytes per stream: each thread produces two adjacent
// states and writes them with one 16-byte store.  Stride seeds use Brown's
// binary skip-ahead only once per thread, from a per-block table of the
// maps of 2^j steps; after that a thread advances to its next pair with
// one precomputed affine map (Q * pairs-per-sweep * 2 steps).
//
// Draws (Eq. 1) are bound by integer issue: the 64-bit state stays in
// registers for all draws of a stream, each step is one 64-bit
// multiply-add (IMAD.WIDE + 2 IMAD), and each uniform is assembled with
// integer instructions (the digest kernel also counts on the fp32 pipe).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "internal.h"
#include "mc_device.cuh"

namespace {

using mcd::Affine;

constexpr int kSeedBlock = 256;
constexpr int kDrawBlock = 256;

// Per-block table of the maps of 2^j LCG steps, j = 0..63 (Brown's squares).
__device__ void build_pow2_table(Affine* tab, uint64_t g, uint64_t c) {
  if (threadIdx.x == 0) {
    Affine sq{g, c};
    for (int j = 0; j < 64; ++j) {
      tab[j] = sq;
      sq = mcd::compose(sq, sq);
    }
  }
  __syncthreads();
}

// The state k steps after x, walking the set bits of k through the table.
__device__ __forceinline__ uint64_t skip_by_table(const Affine* tab, uint64_t x, uint64_t k) {
  while (k) {
    const int j = __ffsll((long long)k) - 1;
    x = mcd::apply(tab[j], x);
    k &= k - 1;
  }
  return x;
}

// The map of k steps, composed from the table.
__device__ __forceinline__ Affine map_by_table(const Affine* tab, uint64_t k) {
  Affine acc{1ull, 0ull};
  while (k) {
    const int j = __ffsll((long long)k) - 1;
    acc = mcd::compose(tab[j], acc);
    k &= k - 1;
  }
  return acc;
}

// ------------------------------------------------------------ hash seeding
template <bool VEC>
__global__ void __launch_bounds__(kSeedBlock) seed_hash_kernel(uint64_t parent_seed, uint64_t key_begin,
                                                               uint64_t count, uint64_t mask,
                                                               uint64_t* __restrict__ out) {
  const uint64_t seed_hash = mcd::seed_hash_of(parent_seed);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (VEC) {
    const uint64_t npairs = count >> 1;
    for (uint64_t p = tid; p < npairs; p += nthreads) {
      const uint64_t k = key_begin + 2 * p;
      ulonglong2 v;
      v.x = mcd::hash_with(k, seed_hash) & mask;
      v.y = mcd::hash_with(k + 1, seed_hash) & mask;
      reinterpret_cast<ulonglong2*>(out)[p] = v;
    }
    if ((count & 1) && tid == 0) out[count - 1] = mcd::hash_with(key_begin + count - 1, seed_hash) & mask;
  } else {
    for (uint64_t i = tid; i < count; i += nthreads) out[i] = mcd::hash_with(key_begin + i, seed_hash) & mask;
  }
}

// ---------------------------------------------------------- stride seeding
template <bool VEC>
__global__ void __launch_bounds__(kSeedBlock) seed_stride_kernel(uint64_t g, uint64_t c, uint64_t x0,
                                                                 uint64_t q, uint64_t id_begin,
                                                                 uint64_t count, uint64_t mask,
                                                                 uint64_t* __restrict__ out) {
  __shared__ Affine tab[64];
  build_pow2_table(tab, g, c);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  if constexpr (VEC) {
    const uint64_t npairs = count >> 1;
    if (tid < npairs) {
      // Unit k = id_begin + 2p gets X_{Qk}; its neighbour is one map of Q steps on.
      const Affine step_q = map_by_table(tab, q);
      const Affine sweep = map_by_table(tab, q * 2ull * nthreads);
      uint64_t x = skip_by_table(tab, x0, q * (id_begin + 2ull * tid));
      for (uint64_t p = tid; p < npairs; p += nthreads) {
        ulonglong2 v;
        v.x = x & mask;
        v.y = mcd::apply(step_q, x) & mask;
        reinterpret_cast<ulonglong2*>(out)[p] = v;
        x = mcd::apply(sweep, x);
      }
    }
    if ((count & 1) && tid == 0)
      out[count - 1] = skip_by_table(tab, x0, q * (id_begin + count - 1)) & mask;
  } else {
    if (tid < count) {
      const Affine sweep = map_by_table(tab, q * nthreads);
      uint64_t x = skip_by_table(tab, x0, q * (id_begin + tid));
      for (uint64_t i = tid; i < count; i += nthreads) {
        out[i] = x & mask;
        x = mcd::apply(sweep, x);
      }
    }
  }
}

// ------------------------------------------------------------------- draws
enum SeedMode { kLoad = 0, kHash = 1, kStride = 2 };

struct DrawArgs {
  uint64_t g, c, mask;
  uint32_t m, draws;
  uint64_t n;
  uint64_t id_begin;
  uint64_t seed, key;  // kHash: global seed s; hierarchical key i (if hier)
  uint32_t hier;       // kHash: 1 = parent seed is hash(key, seed) (Eq. 4)
  uint64_t x0, q;      // kStride
  uint64_t* states;    // kLoad: in/out; else nullable out
  double* u;           // nullable, [draws][n]
  uint64_t* digest;    // nullable, [n]
  // kStride digest kernel: the maps of Q T and 2 Q T steps (T = threads in
  // the grid), the same for every thread; set by the launcher so that they
  // stay in the parameter bank instead of registers
  Affine half, sweep;
};

template <int M, int SEED, bool WANT_U, bool WANT_DIGEST>
__global__ void __launch_bounds__(kDrawBlock) draw_kernel(const DrawArgs a) {
  __shared__ Affine tab[64];
  if constexpr (SEED == kStride) build_pow2_table(tab, a.g, a.c);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  if (tid >= a.n) return;
  Affine sweep{1ull, 0ull};
  uint64_t xs = 0, seed_hash = 0;
  if constexpr (SEED == kHash) seed_hash = mcd::seed_hash_of(a.hier ? mcd::hash64(a.key, a.seed) : a.seed);
  if constexpr (SEED == kStride) {
    sweep = map_by_table(tab, a.q * nthreads);
    xs = skip_by_table(tab, a.x0, a.q * (a.id_begin + tid));
  }
  const uint64_t g = a.g, c = a.c;
  for (uint64_t i = tid; i < a.n; i += nthreads) {
    uint64_t x;
    if constexpr (SEED == kLoad) {
      x = a.states[i];
    } else if constexpr (SEED == kHash) {
      x = mcd::hash_with(a.id_begin + i, seed_hash) & a.mask;
    } else {
      x = xs & a.mask;
      xs = mcd::apply(sweep, xs);
    }
    uint64_t dg = 0;
    double* up = WANT_U ? a.u + i : nullptr;
    uint32_t j = 0;
#pragma unroll 1
    for (; a.draws - j >= 8; j += 8) {  // j <= draws: no wrap near 2^32
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        x = mcd::lcg_step(x, g, c);
        const double v = mcd::u01<M>(x, a.m);
        if constexpr (WANT_DIGEST) dg += mcd::dbits(v);
        if constexpr (WANT_U) {
          __stcs(up, v);
          up += a.n;
        }
      }
    }
    for (; j < a.draws; ++j) {
      x = mcd::lcg_step(x, g, c);
      const double v = mcd::u01<M>(x, a.m);
      if constexpr (WANT_DIGEST) dg += mcd::dbits(v);
      if constexpr (WANT_U) {
        __stcs(up, v);
        up += a.n;
      }
    }
    if (a.states) a.states[i] = x & a.mask;
    if constexpr (WANT_DIGEST) a.digest[i] = dg;
  }
}

// Digest-only draws for m = 63, the integer-issue-bound hot loop.  Each
// thread carries two streams (i and i + T, T = threads in the grid) for
// instruction-level parallelism.  A stream runs on the doubled state
// z = 2x (mod 2^64), the same recurrence with increment 2c, so that the 53
// uniform bits sit at the top of the word.  Per draw: the LCG step
// (IMAD.WIDE + 2 IMAD), the normalising shift s (one bfind), n << s as two
// words (four shifts), s summed on the otherwise idle fp32 pipe; two draws
// share one 64-bit add.  The digest is the sum of the draws' fp64 bit
// patterns, sum(n << s) + (1021 D - sum s) 2^52 (mod 2^64), and equals the
// per-draw sum of dbits(u01_m63(x)).  A stream whose count sum came out NaN
// met a draw with z_hi = 0 (probability 2^-32 per draw) and is redone with
// the exact per-draw path.  DRAWS > 0 fixes the draw count at compile time
// (fully unrolled); DRAWS = 0 reads it at run time and folds the fp32 count
// into an integer every 16 draws, so that it stays exact.  The launch bounds
// are explicit (at least 4 blocks per SM for stride seeds, 1 otherwise):
// they change the compiler's register allocation and schedule, and measured
// 1.73 / 1.80 ms per launch (hash / stride) against 1.78 / 1.87 ms with
// the bare block size.
template <int SEED, int DRAWS>
__global__ void __launch_bounds__(kDrawBlock, SEED == kStride ? 4 : 1) draw_digest_m63_kernel(const DrawArgs a) {
  static_assert(DRAWS % 2 == 0 && DRAWS * 31 < (1 << 24), "count sum must stay exact");
  __shared__ Affine tab[64];
  if constexpr (SEED == kStride) build_pow2_table(tab, a.g, a.c);
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  if (tid >= a.n) return;
  const uint32_t draws = DRAWS > 0 ? (uint32_t)DRAWS : a.draws;
  uint64_t xs = 0, seed_hash = 0;
  if constexpr (SEED == kHash) seed_hash = mcd::seed_hash_of(a.hier ? mcd::hash64(a.key, a.seed) : a.seed);
  if constexpr (SEED == kStride) xs = skip_by_table(tab, a.x0, a.q * (a.id_begin + tid));
  const uint64_t g = a.g, c2 = 2ull * a.c;
  for (uint64_t i = tid; i < a.n; i += 2 * nthreads) {
    const uint64_t i2 = i + nthreads;
    const bool two = i2 < a.n;
    // Starting state (masked) of stream q; called again by the redo.
    auto start = [&](int q) -> uint64_t {
      const uint64_t iq = q == 0 ? i : (two ? i2 : i);
      if constexpr (SEED == kLoad) {
        return a.states[iq];
      } else if constexpr (SEED == kHash) {
        return mcd::hash_with(a.id_begin + iq, seed_hash) & a.mask;
      } else {
        return (q == 0 ? xs : mcd::apply(a.half, xs)) & a.mask;
      }
    };
    uint64_t z[2] = {start(0) << 1, start(1) << 1};
    uint64_t acc[2] = {0ull, 0ull};
    float cnt[2] = {0.f, 0.f};
    uint32_t sum_s[2] = {0u, 0u}, marked = 0u;
    auto fold = [&](int q) {  // run-time count: fp32 partial into the integer sum
      const uint32_t p = __float_as_uint(cnt[q]);
      marked |= mcd::count_marked(cnt[q]) ? (1u << q) : 0u;
      sum_s[q] += p;
      cnt[q] = 0.f;
    };
    if constexpr (DRAWS > 0) {
#pragma unroll
      for (int t = 0; t < DRAWS; t += 2) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          uint64_t y[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            z[q] = g * z[q] + c2;
            const uint32_t s = mcd::clz_or_ones((uint32_t)(z[q] >> 32));
            cnt[q] = mcd::add_count(cnt[q], s);
            y[h] = mcd::n_shifted_m63(z[q], s);
          }
          acc[q] += y[0] + y[1];
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) fold(q);
    } else {
      uint32_t j = 0;
#pragma unroll 1
      for (; draws - j >= 16; j += 16) {  // j <= draws: no wrap near 2^32
#pragma unroll
        for (int t = 0; t < 16; t += 2) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            uint64_t y[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              z[q] = g * z[q] + c2;
              const uint32_t s = mcd::clz_or_ones((uint32_t)(z[q] >> 32));
              cnt[q] = mcd::add_count(cnt[q], s);
              y[h] = mcd::n_shifted_m63(z[q], s);
            }
            acc[q] += y[0] + y[1];
          }
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) fold(q);
      }
      for (; j < draws; ++j) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          z[q] = g * z[q] + c2;
          const uint32_t s = mcd::clz_or_ones((uint32_t)(z[q] >> 32));
          cnt[q] = mcd::add_count(cnt[q], s);
          acc[q] += mcd::n_shifted_m63(z[q], s);
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) fold(q);
    }
    uint64_t x[2], d[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      x[q] = z[q] >> 1;  // the final state mod 2^63
      d[q] = acc[q] + ((uint64_t)((1021u * draws - sum_s[q]) & 0xfffu) << 52);
      if (marked & (1u << q)) {  // exact redo of stream q
        uint64_t xr = start(q), dr = 0;
        for (uint32_t k = 0; k < draws; ++k) {
          xr = mcd::lcg_step(xr, g, a.c);
          dr += mcd::dbits(mcd::u01_m63(xr));
        }
        x[q] = xr & a.mask;
        d[q] = dr;
      }
    }
    if (a.states) a.states[i] = x[0];
    if (a.digest) a.digest[i] = d[0];
    if (two) {
      if (a.states) a.states[i2] = x[1];
      if (a.digest) a.digest[i2] = d[1];
    }
    if constexpr (SEED == kStride) xs = mcd::apply(a.sweep, xs);
  }
}

// Persistent grid: every SM filled to its occupancy limit, never more
// blocks than the work needs.
template <typename K>
int persistent_grid(K kernel, int block, size_t smem, uint64_t work_items) {
  static std::atomic<int> cached[64];  // SM count per device ordinal (0: not read yet)
  int dev = 0;
  cudaGetDevice(&dev);
  int sms = dev >= 0 && dev < 64 ? cached[dev].load(std::memory_order_relaxed) : 0;
  if (sms == 0) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64) cached[dev].store(sms, std::memory_order_relaxed);
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
  if (per_sm < 1) per_sm = 1;
  uint64_t want = (work_items + block - 1) / block;
  uint64_t full = (uint64_t)sms * per_sm;
  if (want < 1) want = 1;
  return (int)(want < full ? want : full);
}

template <int SEED, int DRAWS>
void launch_digest_k(DrawArgs a, cudaStream_t s) {
  auto k = draw_digest_m63_kernel<SEED, DRAWS>;
  const int grid = persistent_grid(k, kDrawBlock, 0, (a.n + 1) / 2);
  if constexpr (SEED == kStride) {
    const uint64_t nthreads = (uint64_t)grid * kDrawBlock;
    a.half = mcd::skip_map(a.g, a.c, a.q * nthreads);
    a.sweep = mcd::skip_map(a.g, a.c, a.q * 2ull * nthreads);
  }
  k<<<grid, kDrawBlock, 0, s>>>(a);
}

template <int SEED>
int launch_digest_m63(const DrawArgs& a, cudaStream_t s) {
  if (a.draws == 64) launch_digest_k<SEED, 64>(a, s);
  else launch_digest_k<SEED, 0>(a, s);
  return mci::cuda_status(cudaGetLastError(), "draw_digest_m63_kernel launch");
}

template <int M, int SEED>
int launch_draw(const DrawArgs& a, cudaStream_t s) {
  const bool wu = a.u != nullptr, wd = a.digest != nullptr;
  if (wu && wd) {
    auto k = draw_kernel<M, SEED, true, true>;
    k<<<persistent_grid(k, kDrawBlock, 0, a.n), kDrawBlock, 0, s>>>(a);
  } else if (wu) {
    auto k = draw_kernel<M, SEED, true, false>;
    k<<<persistent_grid(k, kDrawBlock, 0, a.n), kDrawBlock, 0, s>>>(a);
  } else if (wd) {
    auto k = draw_kernel<M, SEED, false, true>;
    k<<<persistent_grid(k, kDrawBlock, 0, a.n), kDrawBlock, 0, s>>>(a);
  } else {
    auto k = draw_kernel<M, SEED, false, false>;
    k<<<persistent_grid(k, kDrawBlock, 0, a.n), kDrawBlock, 0, s>>>(a);
  }
  return mci::cuda_status(cudaGetLastError(), "draw_kernel launch");
}

template <int M>
int launch_draw_m(const DrawArgs& a, int seed, cudaStream_t s) {
  switch (seed) {
    case kLoad: return launch_draw<M, kLoad>(a, s);
    case kHash: return launch_draw<M, kHash>(a, s);
    default: return launch_draw<M, kStride>(a, s);
  }
}

}  // namespace

extern "C" {

MC_API int mc_seed_hash(mc_ctx* ctx, const mc_lcg* lcg, uint64_t parent_seed, uint64_t key_begin,
                        uint64_t count, uint64_t* d_states, void* stream) {
  if (!ctx) { mci::set_error("mc_seed_hash: ctx is NULL"); return MC_ERR_ARG; }
  int st = mci::check_lcg(lcg);
  if (st != MC_OK) return st;
  if (count == 0) return MC_OK;
  if (!d_states || ((uintptr_t)d_states & 7u)) {
    mci::set_error("mc_seed_hash: d_states is NULL or not 8-byte aligned");
    return MC_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t sh = parent_seed, mask = mcd::mask_of(lcg->m);
  if (((uintptr_t)d_states & 15u) == 0) {
    auto k = seed_hash_kernel<true>;
    k<<<persistent_grid(k, kSeedBlock, 0, (count + 1) / 2), kSeedBlock, 0, s>>>(sh, key_begin, count, mask,
                                                                                  d_states);
  } else {
    auto k = seed_hash_kernel<false>;
    k<<<persistent_grid(k, kSeedBlock, 0, count), kSeedBlock, 0, s>>>(sh, key_begin, count, mask, d_states);
  }
  return mci::cuda_status(cudaGetLastError(), "seed_hash_kernel launch");
}

MC_API int mc_seed_stride(mc_ctx* ctx, const mc_lcg* lcg, uint64_t x0, uint64_t stride_q,
                          uint64_t id_begin, uint64_t count, uint64_t* d_states, void* stream) {
  if (!ctx) { mci::set_error("mc_seed_stride: ctx is NULL"); return MC_ERR_ARG; }
  int st = mci::check_lcg(lcg);
  if (st != MC_OK) return st;
  if (count == 0) return MC_OK;
  if (!d_states || ((uintptr_t)d_states & 7u)) {
    mci::set_error("mc_seed_stride: d_states is NULL or not 8-byte aligned");
    return MC_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t mask = mcd::mask_of(lcg->m);
  if (((uintptr_t)d_states & 15u) == 0) {
    auto k = seed_stride_kernel<true>;
    k<<<persistent_grid(k, kSeedBlock, 0, (count + 1) / 2), kSeedBlock, 0, s>>>(lcg->g, lcg->c, x0, stride_q,
                                                                                  id_begin, count, mask, d_states);
  } else {
    auto k = seed_stride_kernel<false>;
    k<<<persistent_grid(k, kSeedBlock, 0, count), kSeedBlock, 0, s>>>(lcg->g, lcg->c, x0, stride_q, id_begin,
                                                                        count, mask, d_states);
  }
  return mci::cuda_status(cudaGetLastError(), "seed_stride_kernel launch");
}

MC_API int mc_lcg_draw(mc_ctx* ctx, const mc_lcg* lcg, const mc_seed_spec* seed, uint64_t id_begin,
                       uint64_t* d_states, uint64_t n_streams, uint32_t draws, double* d_u,
                       uint64_t* d_digest, void* stream) {
  if (!ctx) { mci::set_error("mc_lcg_draw: ctx is NULL"); return MC_ERR_ARG; }
  int st = mci::check_lcg(lcg);
  if (st != MC_OK) return st;
  if (n_streams == 0) return MC_OK;
  if (!seed && !d_states) {
    mci::set_error("mc_lcg_draw: d_states is NULL and no seed spec is given");
    return MC_ERR_ARG;
  }
  if (seed && (seed->reserved != 0 || seed->mode > MC_SEED_HASH_HIER)) {
    mci::set_error("mc_lcg_draw: bad seed spec (mode %u)", seed->mode);
    return MC_ERR_ARG;
  }
  if (((uintptr_t)d_states & 7u) || ((uintptr_t)d_u & 7u) || ((uintptr_t)d_digest & 7u)) {
    mci::set_error("mc_lcg_draw: buffers must be 8-byte aligned");
    return MC_ERR_ARG;
  }
  DrawArgs a{};
  a.g = lcg->g;
  a.c = lcg->c;
  a.m = lcg->m;
  a.mask = mcd::mask_of(lcg->m);
  a.draws = draws;
  a.n = n_streams;
  a.id_begin = id_begin;
  a.states = d_states;
  a.u = d_u;
  a.digest = d_digest;
  int mode = kLoad;
  if (seed) {
    if (seed->mode == MC_SEED_STRIDE) {
      mode = kStride;
      a.x0 = seed->seed;
      a.q = seed->stride_q;
    } else {
      mode = kHash;
      a.seed = seed->seed;
      a.key = seed->key;
      a.hier = seed->mode == MC_SEED_HASH_HIER ? 1u : 0u;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (lcg->m == 63 && !d_u) {
    // integer-issue-bound form: no uniforms stored, digest and/or final states
    switch (mode) {
      case kLoad: return launch_digest_m63<kLoad>(a, s);
      case kHash: return launch_digest_m63<kHash>(a, s);
      default: return launch_digest_m63<kStride>(a, s);
    }
  }
  if (lcg->m == 63) return launch_draw_m<63>(a, mode, s);
  return launch_draw_m<0>(a, mode, s);
}

}  // extern "C"

// pulse.cu -- the supercritical, time-dependent pulse problem of Section 5:
// a pulse at t = x = 0 in an infinite homogeneous medium, scattering with
// multiplicity (k = c * nu > 1), census at t_end, and the collision-estimator
// flux averaged over [-x_half, x_half] in unit time bins, tallied per
// (repetition, batch).
//
// History-based: a lane follows one source particle and its whole family of
// secondaries depth-first.  Secondaries wait on a per-lane last-in first-out
// stack (thread-local memory).  In hash mode each secondary owns a stream
// seeded on demand by S_c = hash(k, S_p) (Section 4, Eq. 5), so no lane ever
// coordinates with another; in stride mode the family shares the source
// particle's stream, which fixes the depth-first order the secondaries are
// drawn in -- the sequential bookkeeping the paper's hashing removes.
// The fp64 arithmetic is rounded once per operation (--fmad=false).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "internal.h"
#include "mc_log.cuh"
#include "pulse.cuh"
#include "slab.cuh"
#include "transport.h"

namespace {

using mcp::Overflow;
using mcp::PulseDev;
using mcp::pulse_seed;

struct PulseArgs {
  const PulseDev* prob;
  uint64_t range_begin, total;
  uint32_t chunk;
  unsigned long long* ticket;
  unsigned long long* tally;
  unsigned long long* counts;
  uint64_t* hist_state;
  uint64_t* hist_draws;
  mcd::Lcg lcg;
  uint64_t event_cap;
  uint32_t stack_depth;            // pending secondaries a lane keeps (<= kStack)
  mcp::StackRec* stack;            // [stack_depth][threads of the launch]
  const Overflow* ovf_in;          // non-null: the work items are overflowed secondaries
  const unsigned long long* ovf_in_count;
  Overflow* ovf_out;               // non-null (hash modes): where secondaries beyond the stack go
  unsigned long long* ovf_out_count;
  uint64_t ovf_cap;
};

__global__ void pulse_prep_kernel(PulseDev* p) {
  if (threadIdx.x == 0) {
    p->inv_st = 1.0 / p->sigma_t;
    p->unit = __double2ll_rn(p->inv_st * mcs::kFix);
    p->seed_hash = mcd::seed_hash_of(p->seed);
    p->c_n = (uint64_t)ceil(p->c * 0x1p53);
    // floor(nu + u) over u = n 2^-53, n < 2^53, is floor(nu) or floor(nu) + 1
    // (nu <= 64) and does not decrease with n: the first n giving the larger
    // value, found with the same fp64 sum the transport definition uses
    const double fl = floor(p->nu);
    uint64_t lo = 0, hi = 1ull << 53;
    while (lo < hi) {
      const uint64_t mid = lo + ((hi - lo) >> 1);
      if (floor(p->nu + (double)mid * 0x1p-53) > fl) hi = mid;
      else lo = mid + 1;
    }
    p->nu_n = lo;
    p->nu_floor = (uint32_t)fl;
  }
}

struct PulseCounts {
  uint64_t src, flights, coll, absn, scat, census, children, capped, dropped, draws, exh, exd, maxd;
  __device__ void flush(unsigned long long* c) {
    if (src) atomicAdd(c + MC_C_SOURCE, (unsigned long long)src);
    if (flights) atomicAdd(c + MC_C_FLIGHTS, (unsigned long long)flights);
    if (coll) atomicAdd(c + MC_C_COLLISIONS, (unsigned long long)coll);
    if (absn) atomicAdd(c + MC_C_ABSORPTIONS, (unsigned long long)absn);
    if (scat) atomicAdd(c + MC_C_SCATTERS, (unsigned long long)scat);
    if (census) atomicAdd(c + MC_C_LEAK_HI, (unsigned long long)census);
    if (children) atomicAdd(c + MC_C_CHILDREN, (unsigned long long)children);
    if (capped) atomicAdd(c + MC_C_CAPPED, (unsigned long long)capped);
    if (dropped) atomicAdd(c + MC_C_DROPPED, (unsigned long long)dropped);
    if (draws) atomicAdd(c + MC_C_DRAWS, (unsigned long long)draws);
    if (exh) atomicAdd(c + MC_C_EXCEED_HIST, (unsigned long long)exh);
    if (exd) atomicAdd(c + MC_C_EXCEED_DRAWS, (unsigned long long)exd);
    if (maxd) atomicMax(c + MC_C_MAX_DRAWS, (unsigned long long)maxd);
  }
  // The same for a whole converged warp: the counters share a cache line, so
  // the warp's totals go out through one lane.
  __device__ void flush_warp(unsigned long long* c) {
    src = mcd::warp_sum64(src);
    flights = mcd::warp_sum64(flights);
    coll = mcd::warp_sum64(coll);
    absn = mcd::warp_sum64(absn);
    scat = mcd::warp_sum64(scat);
    census = mcd::warp_sum64(census);
    children = mcd::warp_sum64(children);
    capped = mcd::warp_sum64(capped);
    dropped = mcd::warp_sum64(dropped);
    draws = mcd::warp_sum64(draws);
    exh = mcd::warp_sum64(exh);
    exd = mcd::warp_sum64(exd);
    maxd = mcd::warp_max64(maxd);
    if ((threadIdx.x & 31u) == 0u) flush(c);
  }
};

template <int M, bool HASH, bool AGG>
__global__ void __launch_bounds__(256) pulse_kernel(const PulseArgs a) {
  __shared__ mcd::Affine tab[64];
  __shared__ PulseDev sP;
  if (threadIdx.x == 0) {
    mcd::Affine sq{a.lcg.g, a.lcg.c};
    for (int j = 0; j < 64; ++j) { tab[j] = sq; sq = mcd::compose(sq, sq); }
    sP = *a.prob;
  }
  __syncthreads();
  const PulseDev& P = sP;
  const mcd::Lcg l = a.lcg;
  constexpr bool hash_mode = HASH;  // (P.seeding != MC_SEED_STRIDE, chosen by the host)
  const unsigned kFull = 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;

  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  mcp::StackRec* const my_stack = a.stack + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t sp = 0;
  uint64_t pool_next = 0, pool_end = 0;
  bool more = true, alive = false, primary = false;
  PulseCounts lc{};
  mcs::Rng<M> r{0ull, 0ull};
  double x = 0.0, t = 0.0, mu = 0.0;
  uint64_t gi = 0, events = 0, fam_draws = 0;
  uint32_t grp = 0;
  unsigned long long* row = nullptr;
  const uint64_t total = a.ovf_in ? min((uint64_t)*a.ovf_in_count, a.ovf_cap) : a.total;

  for (;;) {
    unsigned dead = __ballot_sync(kFull, !alive);
    while (dead != 0u && more) {
      if (pool_next >= pool_end) {
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(a.ticket, (unsigned long long)a.chunk);
        b0 = __shfl_sync(kFull, b0, 0);
        if (b0 >= total) { more = false; break; }
        pool_next = b0;
        pool_end = min((uint64_t)b0 + (uint64_t)a.chunk, total);
      }
      const uint64_t avail = pool_end - pool_next;
      const unsigned rank = __popc(dead & lt_mask);
      if (!alive && rank < avail && a.ovf_in) {
        // an overflowed secondary: hash seeded, it starts a family of its own
        const Overflow e = a.ovf_in[pool_next + rank];
        grp = e.group;
        row = a.tally + P.tally_offset + (uint64_t)grp * P.n_time_bins;
        r = mcs::Rng<M>{e.seed, 0ull};
        x = e.x;
        t = e.t;
        mu = mcx::two_u_minus_1(r.next_n(l));
        events = 0;
        fam_draws = 0;
        sp = 0;
        primary = false;
        alive = true;
      } else if (!alive && rank < avail) {
        gi = a.range_begin + pool_next + rank;
        grp = (uint32_t)(gi / P.per_batch);
        row = a.tally + P.tally_offset + (uint64_t)grp * P.n_time_bins;
        r = mcs::Rng<M>{pulse_seed(P, gi, tab, l.mask), 0ull};
        x = 0.0;
        t = 0.0;
        mu = mcx::two_u_minus_1(r.next_n(l));
        events = 0;
        fam_draws = 0;
        sp = 0;
        primary = true;
        ++lc.src;
        alive = true;
      }
      pool_next += min((uint64_t)__popc(dead), avail);
      dead = __ballot_sync(kFull, !alive);
    }
    if (__ballot_sync(kFull, alive) == 0u) break;
    if (!alive) continue;

    bool ended = false, redraw = false;
    if (events == a.event_cap) {
      ++lc.capped;
      ended = true;
    } else {
      ++events;
      ++lc.flights;
      const double d = -mclog::log1m_n(r.next_n(l)) * P.inv_st;
      const double tn = t + d;
      if (!mcs::nn_lt(tn, P.t_end)) {  // tn >= t_end, both non-negative
        ++lc.census;
        ended = true;
      } else {
        const double xn = x + d * mu;
        ++lc.coll;
        if (mcx::abs_le(xn, P.x_half)) {
          const uint64_t jf = mcx::floor_nonneg(tn);
          const uint32_t j = jf < P.n_time_bins ? (uint32_t)jf : P.n_time_bins - 1;
          if constexpr (AGG) mcd::warp_agg_add(row + j, (unsigned long long)P.unit);
          else atomicAdd(row + j, (unsigned long long)P.unit);
        }
        x = xn;
        t = tn;
        if (r.next_n(l) < P.c_n) {  // u < c
          ++lc.scat;
          const uint32_t n = P.nu_floor + (r.next_n(l) >= P.nu_n ? 1u : 0u);  // floor(nu + u)
          for (uint32_t k = 0; k + 1 < n; ++k) {
            const uint64_t seed = hash_mode ? (mcd::hash64((uint64_t)k, r.x & l.mask) & l.mask) : 0ull;
            if (sp < a.stack_depth) {
              mcp::stack_put(my_stack + sp * nthreads, x, t, seed);
              ++sp;
              ++lc.children;
            } else if (a.ovf_out) {  // hash modes only
              const unsigned long long idx = atomicAdd(a.ovf_out_count, 1ull);
              if (idx < a.ovf_cap) {
                a.ovf_out[idx] = Overflow{x, t, seed, grp, 0u};
                ++lc.children;
              } else {
                ++lc.dropped;
              }
            } else {
              ++lc.dropped;  // reported as MC_ERR_CAPACITY by mc_tally_read
            }
          }
          // its new direction: drawn in place (hash) or below, on the code path the
          // pop shares (stride; measured faster for each variant)
          if constexpr (HASH) mu = mcx::two_u_minus_1(r.next_n(l));
          else redraw = true;
        } else {
          ++lc.absn;
          ended = true;
        }
      }
    }
    if (ended) {  // the current particle ended
      if (hash_mode) {
        fam_draws += r.draws;
        if (r.draws > lc.maxd) lc.maxd = r.draws;
        if (primary) {
          if (a.hist_state) a.hist_state[gi] = r.x & l.mask;
          if (a.hist_draws) a.hist_draws[gi] = r.draws;
          if (P.stride_q != 0 && r.draws > P.stride_q) { ++lc.exh; lc.exd += r.draws - P.stride_q; }
        }
      }
      primary = false;
      events = 0;
      if (sp > 0) {  // the next secondary of the family; its direction below
        --sp;
        uint64_t seed;
        mcp::stack_get(my_stack + sp * nthreads, x, t, seed);
        if constexpr (HASH) {
          r = mcs::Rng<M>{seed, 0ull};
          mu = mcx::two_u_minus_1(r.next_n(l));
        } else {
          redraw = true;
        }
      } else {
        if (!hash_mode) {
          fam_draws = r.draws;
          if (r.draws > lc.maxd) lc.maxd = r.draws;
          if (a.hist_state) a.hist_state[gi] = r.x & l.mask;
          if (a.hist_draws) a.hist_draws[gi] = r.draws;
          if (P.stride_q != 0 && r.draws > P.stride_q) { ++lc.exh; lc.exd += r.draws - P.stride_q; }
        }
        lc.draws += fam_draws;
        alive = false;
      }
    }
    // stride: one code path draws the direction of a scattered or a popped
    // particle (the same draw, in the same stream order, as drawing it in place)
    if (redraw) mu = mcx::two_u_minus_1(r.next_n(l));
  }
  lc.flush_warp(a.counts);
}

}  // namespace

namespace mci {

size_t pulse_dev_size() { return sizeof(PulseDev); }

int pulse_fill_host(const mc_problem* src, void* dst) {
  PulseDev q;
  std::memset(&q, 0, sizeof q);
  const mc_pulse_spec* s = src->pulse;
  q.c = s->c;
  q.nu = s->nu;
  q.t_end = s->t_end;
  q.x_half = s->x_half;
  q.sigma_t = s->sigma_t;
  q.n_hist = src->n_histories;
  q.seed = src->seed;
  q.stride_q = src->stride_q;
  q.id_offset = src->id_offset;
  q.tally_offset = src->tally_offset;
  q.n_reps = s->n_reps;
  q.n_batches = s->n_batches;
  q.per_batch = s->per_batch;
  q.n_time_bins = s->n_time_bins;
  q.seeding = src->seeding;
  q.n_census = s->n_census;
  q.pc_target = s->pc_target;
  std::memcpy(dst, &q, sizeof q);
  return MC_OK;
}

int pulse_prep(void* d_prob, cudaStream_t s) {
  pulse_prep_kernel<<<1, 32, 0, s>>>(static_cast<PulseDev*>(d_prob));
  return cuda_status(cudaGetLastError(), "pulse_prep_kernel launch");
}

// The kernel variant for the LCG width, the seeding mode and the tally atomics.
static void (*pulse_kernel_for(uint32_t m, bool hash, bool agg))(const PulseArgs) {
  if (agg) return m == 63 ? (hash ? pulse_kernel<63, true, true> : pulse_kernel<63, false, true>)
                          : (hash ? pulse_kernel<0, true, true> : pulse_kernel<0, false, true>);
  return m == 63 ? (hash ? pulse_kernel<63, true, false> : pulse_kernel<63, false, false>)
                 : (hash ? pulse_kernel<0, true, false> : pulse_kernel<0, false, false>);
}

// The largest grid pulse_run launches for L (one persistent block per slot).
static int pulse_full_grid(const PulseLaunch& L, uint64_t* full_out) {
  const bool hash = L.seeding != MC_SEED_STRIDE;
  auto k = pulse_kernel_for(L.lcg.m, hash, L.tally_agg);
  int per_sm = 0;
  int st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, L.block, 0),
                       "cudaOccupancyMaxActiveBlocksPerMultiprocessor(pulse)");
  if (st != MC_OK) return st;
  if (per_sm < 1) per_sm = 1;
  *full_out = (uint64_t)L.num_sms * per_sm;
  return MC_OK;
}

int pulse_stack_bytes(const PulseLaunch& L, size_t* bytes) {
  uint64_t full = 0;
  const int st = pulse_full_grid(L, &full);
  if (st != MC_OK) return st;
  *bytes = (size_t)full * (size_t)L.block * L.stack_depth * sizeof(mcp::StackRec);
  return MC_OK;
}

int pulse_run(const PulseLaunch& L, cudaStream_t s) {
  PulseArgs a{};
  a.prob = static_cast<const PulseDev*>(L.d_prob);
  a.range_begin = L.range_begin;
  a.total = L.total;
  a.chunk = L.chunk;
  a.ticket = L.d_ticket;
  a.tally = reinterpret_cast<unsigned long long*>(L.tally->d_bins);
  a.counts = reinterpret_cast<unsigned long long*>(L.tally->d_counts);
  a.hist_state = L.tally->d_hist_state;
  a.hist_draws = L.tally->d_hist_draws;
  a.lcg = mcd::Lcg{L.lcg.g, L.lcg.c, mcd::mask_of(L.lcg.m), L.lcg.m};
  a.event_cap = L.event_cap;
  a.stack_depth = L.stack_depth;
  a.stack = static_cast<mcp::StackRec*>(L.d_stack);
  const bool hash = L.seeding != MC_SEED_STRIDE;
  auto k = pulse_kernel_for(L.lcg.m, hash, L.tally_agg);
  uint64_t full = 0;
  int st = pulse_full_grid(L, &full);
  if (st != MC_OK) return st;
  if (!L.d_stack || L.stack_bytes < (size_t)full * L.block * L.stack_depth * sizeof(mcp::StackRec)) {
    set_error("pulse transport: the lane stacks need more device memory than was given");
    return MC_ERR_ARG;
  }
  const uint64_t warps_needed = (a.total + a.chunk - 1) / a.chunk;
  const uint64_t blocks_needed = (warps_needed * 32 + L.block - 1) / L.block;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(full, blocks_needed));
  if (!L.d_ovf) {
    k<<<grid, L.block, 0, s>>>(a);
    return cuda_status(cudaGetLastError(), "pulse_kernel launch");
  }
  // Hash modes: secondaries beyond the lane stacks go to an overflow bank,
  // processed generation by generation until a generation overflows nothing.
  auto* cnt = static_cast<unsigned long long*>(L.d_ovf);
  Overflow* bank[2] = {reinterpret_cast<Overflow*>(static_cast<char*>(L.d_ovf) + 256),
                       reinterpret_cast<Overflow*>(static_cast<char*>(L.d_ovf) + 256 + L.ovf_cap * sizeof(Overflow))};
  a.ovf_cap = L.ovf_cap;
  a.ovf_out = bank[0];
  a.ovf_out_count = cnt;
  MC_TRY_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s));
  k<<<grid, L.block, 0, s>>>(a);
  st = cuda_status(cudaGetLastError(), "pulse_kernel launch");
  for (int gen = 1; st == MC_OK; ++gen) {
    const int cur = (gen - 1) & 1, nxt = cur ^ 1;
    MC_TRY_CUDA(cudaMemcpyAsync(L.h_count, cnt + cur, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    MC_TRY_CUDA(cudaStreamSynchronize(s));
    const uint64_t made = std::min<uint64_t>(*L.h_count, L.ovf_cap);
    if (made == 0) break;
    if ((uint32_t)gen > L.max_generations) {
      set_error("pulse transport: more than %u generations of overflowed secondaries", L.max_generations);
      return MC_ERR_TIMEOUT;
    }
    PulseArgs b = a;
    b.ovf_in = bank[cur];
    b.ovf_in_count = cnt + cur;
    b.ovf_out = bank[nxt];
    b.ovf_out_count = cnt + nxt;
    b.total = made;
    MC_TRY_CUDA(cudaMemsetAsync(cnt + nxt, 0, sizeof(unsigned long long), s));
    MC_TRY_CUDA(cudaMemsetAsync(L.d_ticket, 0, sizeof(unsigned long long), s));
    const uint64_t w = (made + a.chunk - 1) / a.chunk;
    const int g2 = (int)std::max<uint64_t>(1, std::min<uint64_t>(full, (w * 32 + L.block - 1) / L.block));
    k<<<g2, L.block, 0, s>>>(b);
    st = cuda_status(cudaGetLastError(), "pulse_kernel launch (overflow)");
  }
  return st;
}

size_t pulse_ovf_bytes(uint64_t cap) { return 256 + 2 * cap * sizeof(Overflow); }

}  // namespace mci

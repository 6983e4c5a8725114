// pulse_census.cu -- the pulse problem of Section 5 run in census phases,
// with population control by one-off hashed values (Section 4) between
// phases and on-demand seeds for the copies (Eq. 5).
//
// One launch per phase.  A lane takes a work item -- a source history in
// the first phase, a banked particle afterwards -- and follows it, its
// copies and all their secondaries depth-first until each is absorbed or
// reaches the phase's census time.  A particle reaching the census is
// appended to the next bank (one atomic per group of lanes that bank
// together) and its weight, as int64 fixed point, is added to its group's
// total.  The next launch turns each banked particle into
//   n = floor(w N / W + xi),  xi = (hash(2^63 + p, S) >> 11) 2^-53
// copies, with W the group's exact total; xi is a one-off value of the
// particle's own state S.  Because n depends only on the particle and on
// an exact integer sum, the order of the bank -- which atomics make
// nondeterministic -- changes no result: tallies and counters are
// bit-identical to the sequential definition.
//
// The host enqueues the phases back to back (each launch reads the size of
// its input bank from device memory); it waits only to read how many
// secondaries overflowed the lane stacks in a phase, and launches the
// generations of those before the phase's control.
// The fp64 arithmetic is rounded once per operation (--fmad=false).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "mc_log.cuh"
#include "pulse.cuh"
#include "slab.cuh"
#include "transport.h"

namespace cg = cooperative_groups;

namespace {

using mcp::kStack;
using mcp::Overflow;
using mcp::Pending;
using mcp::PulseDev;

// A particle waiting at a census (48 bytes).
struct BankRec {
  double x, mu, w;
  uint64_t s;      // LCG state, masked to m bits
  uint64_t draws;  // draws made from this stream so far
  uint32_t group;  // rep * n_batches + batch
  uint32_t pad;
};

constexpr uint64_t kOneOffKey = 1ull << 63;  // keys of one-off values: 2^63 + phase

// Per group, derived from the group's exact weight total W after a phase:
// the factor N / (W 2^-32) of the copy counts (0 when W = 0: no copies),
// the copies' weight W 2^-32 / N, its collision score and its fixed point.
struct GroupCtl {
  double ratio, w;
  long long unit, wfix;
};

struct CensusArgs {
  const PulseDev* prob;
  uint32_t phase;  // p = 1..C; the launch ends particles at T_p
  int last;        // p == C: the census at T_p ends particles
  double t0, tp;   // T_{p-1}, T_p
  uint64_t range_begin, n_src;  // first phase: source histories
  uint64_t group_begin;         // first group of the range
  const BankRec* in;            // later phases: banked particles
  int stage;                    // bank items staged per chunk in shared memory (chunk <= kPrefetch)
  const unsigned long long* in_count;
  const GroupCtl* ctl;          // per group: control of `in`
  BankRec* out;
  unsigned long long* out_count;
  unsigned long long* w_out;    // per group: exact weight total of `out`
  uint64_t cap;
  uint32_t chunk;
  unsigned long long* ticket;
  unsigned long long* tally;
  unsigned long long* counts;
  mcd::Lcg lcg;
  uint64_t event_cap;
  uint32_t stack_depth;            // pending secondaries a lane keeps (<= kStack)
  const Overflow* ovf_in;          // non-null: the work items are overflowed secondaries
  const unsigned long long* ovf_in_count;
  Overflow* ovf_out;               // where secondaries beyond the stack go
  unsigned long long* ovf_out_count;
  uint64_t ovf_cap;
};

struct CensusCounts {
  uint64_t src, flights, coll, absn, scat, census, children, capped, dropped, draws, maxd, banked, splits, kills;
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
    if (maxd) atomicMax(c + MC_C_MAX_DRAWS, (unsigned long long)maxd);
    if (banked) atomicAdd(c + MC_C_BANKED, (unsigned long long)banked);
    if (splits) atomicAdd(c + MC_C_SPLITS, (unsigned long long)splits);
    if (kills) atomicAdd(c + MC_C_ROULETTE_KILLS, (unsigned long long)kills);
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
    maxd = mcd::warp_max64(maxd);
    banked = mcd::warp_sum64(banked);
    splits = mcd::warp_sum64(splits);
    kills = mcd::warp_sum64(kills);
    if ((threadIdx.x & 31u) == 0u) flush(c);
  }
  __device__ void stream_end(uint64_t d) {
    draws += d;
    if (d > maxd) maxd = d;
  }
};

// Bank items arrive one lane at a time as lanes finish, and each start is
// two dependent loads (the record, then its group's control).  A warp that
// takes a chunk of bank items loads all of its records and their controls
// at once into shared memory (at most kPrefetch items per warp), so the
// chunk pays one round trip instead of one per item.
constexpr uint32_t kPrefetch = 64;  // largest chunk staged
struct StagedItem {
  BankRec e;
  GroupCtl gc;
};

template <int M, bool AGG>
__global__ void __maxnreg__(96) pulse_census_kernel(const CensusArgs a) {
  extern __shared__ StagedItem s_items[];
  __shared__ PulseDev sP;
  if (threadIdx.x == 0) sP = *a.prob;
  __syncthreads();
  const PulseDev& P = sP;
  const mcd::Lcg l = a.lcg;
  const unsigned kFull = 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint64_t total = a.ovf_in ? min((uint64_t)*a.ovf_in_count, a.ovf_cap)
                                  : (a.in ? min((uint64_t)*a.in_count, a.cap) : a.n_src);
  const bool staged = a.stage && a.in != nullptr && a.ovf_in == nullptr;
  uint64_t chunk_base = 0;

  Pending stack[kStack];
  uint32_t sp = 0;
  uint64_t pool_next = 0, pool_end = 0;
  bool more = true, alive = false;
  CensusCounts lc{};
  mcs::Rng<M> r{0ull, 0ull};
  double x = 0.0, t = 0.0, mu = 0.0, w = 1.0;
  double x0 = 0.0, mu0 = 0.0;  // the banked particle whose copies this lane runs
  uint64_t s0 = 0, copies_left = 0, next_key = 0, events = 0;
  long long unit_w = 0, wfix = 0;  // collision score and fixed-point weight of w
  uint32_t grp = 0;
  unsigned long long* row = nullptr;

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
        chunk_base = b0;
        if (staged) {
          // the chunk's records and their group controls, coalesced
          StagedItem* w = s_items + (threadIdx.x >> 5) * a.chunk;
          for (uint64_t j = lane; b0 + j < pool_end; j += 32) {
            const BankRec e = a.in[b0 + j];
            w[j].e = e;
            w[j].gc = a.ctl[e.group - a.group_begin];
          }
          __syncwarp();
        }
      }
      const uint64_t avail = pool_end - pool_next;
      const unsigned rank = __popc(dead & lt_mask);
      if (!alive && rank < avail) {
        const uint64_t item = pool_next + rank;
        if (a.ovf_in) {
          // an overflowed secondary of this phase: the phase's group weight
          const Overflow e = a.ovf_in[item];
          grp = e.group;
          if (a.phase == 1) {
            w = 1.0;
            unit_w = P.unit;
            wfix = (long long)mcs::kFix;
          } else {
            const GroupCtl gc = a.ctl[grp - a.group_begin];
            w = gc.w;
            unit_w = gc.unit;
            wfix = gc.wfix;
          }
          r = mcs::Rng<M>{e.seed, 0ull};
          x = e.x;
          t = e.t;
          mu = mcx::two_u_minus_1(r.next_n(l));
          copies_left = 0;
          alive = true;
        } else if (a.in == nullptr) {
          const uint64_t g = a.range_begin + item;
          grp = (uint32_t)(g / P.per_batch);
          r = mcs::Rng<M>{mcp::pulse_seed(P, g, nullptr, l.mask), 0ull};  // hash modes only
          x = 0.0;
          t = a.t0;
          mu = mcx::two_u_minus_1(r.next_n(l));
          w = 1.0;
          unit_w = P.unit;
          wfix = (long long)mcs::kFix;
          copies_left = 0;
          ++lc.src;
          alive = true;
        } else {
          const StagedItem* si = staged ? s_items + (threadIdx.x >> 5) * a.chunk + (item - chunk_base) : nullptr;
          const BankRec e = staged ? si->e : a.in[item];
          grp = e.group;
          const GroupCtl gc = staged ? si->gc : a.ctl[grp - a.group_begin];
          // xi = h 2^-53 and the floor (of a non-negative sum) on the integer pipes
          const uint64_t h = mcd::hash64(kOneOffKey + (a.phase - 1), e.s) >> 11;
          const double xi = mcd::u53_to_double((uint32_t)(h >> 32), (uint32_t)h);
          const uint64_t n = mcx::floor_nonneg(e.w * gc.ratio + xi);
          if (n == 0) {
            ++lc.kills;
            lc.stream_end(e.draws);
          } else {
            lc.splits += n - 1;
            w = gc.w;
            unit_w = gc.unit;
            wfix = gc.wfix;
            x0 = e.x;
            mu0 = e.mu;
            s0 = e.s;
            copies_left = n - 1;
            next_key = 0;
            r = mcs::Rng<M>{e.s, e.draws};
            x = x0;
            t = a.t0;
            mu = mu0;
            alive = true;
          }
        }
        if (alive) {
          row = a.tally + P.tally_offset + (uint64_t)grp * P.n_time_bins;
          events = 0;
          sp = 0;
        }
      }
      pool_next += min((uint64_t)__popc(dead), avail);
      dead = __ballot_sync(kFull, !alive);
    }
    if (__ballot_sync(kFull, alive) == 0u) break;
    if (!alive) continue;

    bool ended = false, banked = false, redraw = false;
    if (events == a.event_cap) {
      ++lc.capped;
      ended = true;
    } else {
      ++events;
      ++lc.flights;
      const double d = -mclog::log1m_n(r.next_n(l)) * P.inv_st;
      const double tn = t + d;
      if (!mcs::nn_lt(tn, a.tp)) {  // tn >= T_p, both non-negative
        ended = true;
        if (a.last) {
          ++lc.census;
        } else {
          banked = true;
          ++lc.banked;
          BankRec e;
          e.x = x + (a.tp - t) * mu;
          e.mu = mu;
          e.w = w;
          e.s = r.x & l.mask;
          e.draws = r.draws;
          e.group = grp;
          e.pad = 0;
          cg::coalesced_group cgp = cg::coalesced_threads();
          unsigned long long base = 0;
          if (cgp.thread_rank() == 0) base = atomicAdd(a.out_count, (unsigned long long)cgp.size());
          base = cgp.shfl(base, 0);
          const uint64_t idx = base + cgp.thread_rank();
          if (idx < a.cap) a.out[idx] = e;
          else ++lc.dropped;  // reported as MC_ERR_CAPACITY by mc_tally_read
          // lanes of one group carry one weight in a phase: one atomic per group
          cg::coalesced_group same = cg::labeled_partition(cgp, grp);
          if (same.thread_rank() == 0)
            atomicAdd(a.w_out + (grp - a.group_begin), (unsigned long long)(wfix * (long long)same.size()));
        }
      } else {
        const double xn = x + d * mu;
        ++lc.coll;
        if (mcx::abs_le(xn, P.x_half)) {
          const uint64_t jf = mcx::floor_nonneg(tn);
          const uint32_t j = jf < P.n_time_bins ? (uint32_t)jf : P.n_time_bins - 1;
          if constexpr (AGG) mcd::warp_agg_add(row + j, (unsigned long long)unit_w);
          else atomicAdd(row + j, (unsigned long long)unit_w);
        }
        x = xn;
        t = tn;
        if (r.next_n(l) < P.c_n) {  // u < c
          ++lc.scat;
          const uint32_t n = P.nu_floor + (r.next_n(l) >= P.nu_n ? 1u : 0u);  // floor(nu + u)
          for (uint32_t k = 0; k + 1 < n; ++k) {
            const uint64_t seed = mcd::hash64((uint64_t)k, r.x & l.mask) & l.mask;
            if (sp < a.stack_depth) {
              stack[sp].x = x;
              stack[sp].t = t;
              stack[sp].seed = seed;
              ++sp;
              ++lc.children;
            } else {
              const unsigned long long idx = atomicAdd(a.ovf_out_count, 1ull);
              if (idx < a.ovf_cap) {
                a.ovf_out[idx] = Overflow{x, t, seed, grp, 0u};
                ++lc.children;
              } else {
                ++lc.dropped;  // reported as MC_ERR_CAPACITY by mc_tally_read
              }
            }
          }
          redraw = true;  // its new direction, drawn below
        } else {
          ++lc.absn;
          ended = true;
        }
      }
    }
    if (ended) {
      if (!banked) lc.stream_end(r.draws);
      events = 0;
      if (sp > 0) {  // next secondary of this family; its direction below
        --sp;
        x = stack[sp].x;
        t = stack[sp].t;
        r = mcs::Rng<M>{stack[sp].seed, 0ull};
        redraw = true;
      } else if (copies_left > 0) {  // next copy of the banked particle: Eq. (5) seed
        --copies_left;
        r = mcs::Rng<M>{mcd::hash64(next_key, s0) & l.mask, 0ull};
        ++next_key;
        x = x0;
        t = a.t0;
        mu = mu0;
      } else {
        alive = false;
      }
    }
    // one code path draws the direction of a scattered or a popped particle
    if (redraw) mu = mcx::two_u_minus_1(r.next_n(l));
  }
  lc.flush_warp(a.counts);
}

// Control of each group after a phase: GroupCtl from the exact weight
// total, which is then cleared for the next phase.
__global__ void census_control_kernel(const PulseDev* __restrict__ prob, unsigned long long* __restrict__ wsum,
                                      GroupCtl* __restrict__ ctl, uint64_t groups) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= groups) return;
  const double n_target = (double)(prob->pc_target ? prob->pc_target : prob->per_batch);
  const long long W = (long long)wsum[i];
  GroupCtl g{0.0, 0.0, 0, 0};
  if (W > 0) {
    const double wd = (double)W * 0x1p-32;
    g.ratio = n_target / wd;
    g.w = wd / n_target;
    g.unit = __double2ll_rn(g.w * prob->inv_st * mcs::kFix);
    g.wfix = __double2ll_rn(g.w * mcs::kFix);
  }
  ctl[i] = g;
  wsum[i] = 0ull;
}

// Census time T_p: 0, t_end p / C, t_end.
double census_time(const mc_pulse_spec& s, uint32_t p) {
  if (p == 0) return 0.0;
  if (p >= s.n_census) return s.t_end;
  return s.t_end * (double)p / (double)s.n_census;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

namespace mci {

uint64_t pulse_census_cap(const mc_pulse_spec& s, uint64_t groups) {
  const double k = s.c * s.nu;
  const double growth = std::exp(std::max(0.0, k - 1.0) * s.sigma_t * (s.t_end / (double)s.n_census));
  const double per = (double)std::max<uint32_t>(s.per_batch, s.pc_target ? s.pc_target : s.per_batch);
  const double e = (double)groups * per * growth;
  return (uint64_t)std::ceil(1.25 * e + 16.0 * std::sqrt(e)) + 4096;
}

size_t pulse_census_bytes(uint64_t groups, uint64_t cap) {
  return 256 + align256(groups * sizeof(long long)) + align256(groups * sizeof(GroupCtl)) +
         2 * align256(cap * sizeof(BankRec));
}

int pulse_census_run(const PulseCensusLaunch& L, cudaStream_t s) {
  const mc_pulse_spec& spec = *L.spec;
  char* base = static_cast<char*>(L.d_buf);
  auto* cnt = reinterpret_cast<unsigned long long*>(base);
  size_t off = 256;
  auto* wsum = reinterpret_cast<unsigned long long*>(base + off);
  off += align256(L.groups * sizeof(long long));
  auto* ctl = reinterpret_cast<GroupCtl*>(base + off);
  off += align256(L.groups * sizeof(GroupCtl));
  BankRec* bank[2] = {reinterpret_cast<BankRec*>(base + off),
                      reinterpret_cast<BankRec*>(base + off + align256(L.cap * sizeof(BankRec)))};
  auto k = L.base.tally_agg ? (L.base.lcg.m == 63 ? pulse_census_kernel<63, true> : pulse_census_kernel<0, true>)
                            : (L.base.lcg.m == 63 ? pulse_census_kernel<63, false> : pulse_census_kernel<0, false>);
  const int stage = L.base.chunk <= kPrefetch ? 1 : 0;
  const size_t stage_smem = stage ? (size_t)(L.base.block / 32) * L.base.chunk * sizeof(StagedItem) : 0u;
  int per_sm = 0;
  int st = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, L.base.block, stage_smem),
                       "cudaOccupancyMaxActiveBlocksPerMultiprocessor(pulse census)");
  if (st != MC_OK) return st;
  if (per_sm < 1) per_sm = 1;
  const uint64_t full = (uint64_t)L.base.num_sms * (uint64_t)per_sm;

  CensusArgs a{};
  a.prob = static_cast<const PulseDev*>(L.base.d_prob);
  a.range_begin = L.base.range_begin;
  a.n_src = L.base.total;
  a.group_begin = L.group_begin;
  a.cap = L.cap;
  a.chunk = L.base.chunk;
  a.ticket = L.base.d_ticket;
  a.tally = reinterpret_cast<unsigned long long*>(L.base.tally->d_bins);
  a.counts = reinterpret_cast<unsigned long long*>(L.base.tally->d_counts);
  a.lcg = mcd::Lcg{L.base.lcg.g, L.base.lcg.c, mcd::mask_of(L.base.lcg.m), L.base.lcg.m};
  a.event_cap = L.base.event_cap;
  a.stack_depth = L.base.stack_depth;
  a.stage = stage;
  auto* ocnt = static_cast<unsigned long long*>(L.base.d_ovf);
  Overflow* obank[2] = {
      reinterpret_cast<Overflow*>(static_cast<char*>(L.base.d_ovf) + 256),
      reinterpret_cast<Overflow*>(static_cast<char*>(L.base.d_ovf) + 256 + L.base.ovf_cap * sizeof(Overflow))};
  a.ovf_cap = L.base.ovf_cap;
  const uint32_t C = spec.n_census;
  MC_TRY_CUDA(cudaMemsetAsync(wsum, 0, L.groups * sizeof(long long), s));
  for (uint32_t p = 1; p <= C; ++p) {
    const int out = (int)((p - 1) & 1u), in = out ^ 1;
    a.phase = p;
    a.last = p == C;
    a.t0 = census_time(spec, p - 1);
    a.tp = census_time(spec, p);
    a.in = p == 1 ? nullptr : bank[in];
    a.in_count = cnt + in;
    a.ctl = ctl;
    a.out = bank[out];
    a.out_count = cnt + out;
    a.w_out = wsum;
    MC_TRY_CUDA(cudaMemsetAsync(L.base.d_ticket, 0, sizeof(unsigned long long), s));
    if (!a.last) MC_TRY_CUDA(cudaMemsetAsync(cnt + out, 0, sizeof(unsigned long long), s));
    uint64_t grid = full;
    if (p == 1) {
      const uint64_t warps = (a.n_src + a.chunk - 1) / a.chunk;
      grid = std::max<uint64_t>(1, std::min<uint64_t>(full, (warps * 32 + L.base.block - 1) / L.base.block));
    }
    a.ovf_in = nullptr;
    a.ovf_out = obank[0];
    a.ovf_out_count = ocnt;
    MC_TRY_CUDA(cudaMemsetAsync(ocnt, 0, 2 * sizeof(unsigned long long), s));
    k<<<(int)grid, L.base.block, p == 1 ? 0u : stage_smem, s>>>(a);
    st = cuda_status(cudaGetLastError(), "pulse_census_kernel launch");
    if (st != MC_OK) return st;
    // secondaries that overflowed the lane stacks, generation by generation
    for (int gen = 1;; ++gen) {
      const int cur = (gen - 1) & 1, nxt = cur ^ 1;
      MC_TRY_CUDA(cudaMemcpyAsync(L.base.h_count, ocnt + cur, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                  s));
      MC_TRY_CUDA(cudaStreamSynchronize(s));
      if (*L.base.h_count == 0) break;
      if ((uint32_t)gen > L.base.max_generations) {
        set_error("pulse census: more than %u generations of overflowed secondaries", L.base.max_generations);
        return MC_ERR_TIMEOUT;
      }
      CensusArgs b = a;
      b.ovf_in = obank[cur];
      b.ovf_in_count = ocnt + cur;
      b.ovf_out = obank[nxt];
      b.ovf_out_count = ocnt + nxt;
      MC_TRY_CUDA(cudaMemsetAsync(ocnt + nxt, 0, sizeof(unsigned long long), s));
      MC_TRY_CUDA(cudaMemsetAsync(L.base.d_ticket, 0, sizeof(unsigned long long), s));
      const uint64_t made = std::min<uint64_t>(*L.base.h_count, L.base.ovf_cap);
      const uint64_t w = (made + a.chunk - 1) / a.chunk;
      const uint64_t g2 = std::max<uint64_t>(1, std::min<uint64_t>(full, (w * 32 + L.base.block - 1) / L.base.block));
      k<<<(int)g2, L.base.block, 0, s>>>(b);
      st = cuda_status(cudaGetLastError(), "pulse_census_kernel launch (overflow)");
      if (st != MC_OK) return st;
    }
    if (!a.last) {
      census_control_kernel<<<(unsigned)((L.groups + 255) / 256), 256, 0, s>>>(a.prob, wsum, ctl, L.groups);
      st = cuda_status(cudaGetLastError(), "census_control_kernel launch");
      if (st != MC_OK) return st;
    }
  }
  return MC_OK;
}

}  // namespace mci

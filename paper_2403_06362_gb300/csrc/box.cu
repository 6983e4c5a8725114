// box.cu -- history-based transport of the two-region multigroup box.
//
// A persistent kernel with lane refill (as for the slab) follows one
// particle per lane.  Work items are either source histories (a ticket over
// global history indices) or the split children waiting in a device bank.
// Children created by a launch are appended to the other bank; the host then
// launches the next generation on them, until a generation creates none.
// Every particle's stream depends only on its own seed (Eq. 3/4 for sources,
// Eq. 5 for children), so the generation order changes no result, and the
// int64 mesh tally is bit-identical to any other schedule.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "box.cuh"
#include "internal.h"
#include "transport.h"

namespace {

using mcb::BoxDev;
using mcb::ChildRec;

__global__ void box_prep_kernel(BoxDev* __restrict__ p, uint32_t n) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    BoxDev& b = p[i];
    b.h = b.side / (double)b.mesh;
    b.inv_h = (double)b.mesh / b.side;
    mcx::fixed_of(b.inv_h, b.ih_q, b.ih_s);
    b.side_f = (float)b.side;
    b.lo_f = (float)b.lo;
    b.hi_f = (float)b.hi;
    b.h_f = b.side_f / (float)b.mesh;
    b.inv_h_f = (float)b.mesh / b.side_f;
    for (int r = 0; r < 2; ++r) {
      b.inv_st[r] = 1.0 / b.st[r];
      b.inv_st_f[r] = 1.0f / (float)b.st[r];
      b.c_f[r] = (float)b.c[r];
      b.wl_f[r] = (float)b.wl[r];
      b.wh_f[r] = (float)b.wh[r];
      b.ws_f[r] = (float)b.ws[r];
    }
    const uint64_t parent = b.seeding == MC_SEED_HASH_HIER ? mcd::hash64(b.key, b.seed) : b.seed;
    b.seed_hash = mcd::seed_hash_of(parent);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t acc = 0;
    for (uint32_t i = 0; i < n; ++i) {
      p[i].hist_begin = acc;
      acc += p[i].n_hist;
    }
  }
}

struct BoxArgs {
  const BoxDev* probs;
  uint32_t nprob;
  uint32_t chunk;
  const ChildRec* child_in;  // nullptr: the work items are source histories
  uint64_t range_begin, total;
  unsigned long long* ticket;
  ChildRec* child_out;
  unsigned long long* child_out_count;
  uint64_t child_cap;
  unsigned long long* tally;
  unsigned long long* counts;
  uint64_t* hist_state;
  uint64_t* hist_draws;
  mcd::Lcg lcg;
  uint64_t event_cap;
};

__device__ __forceinline__ uint32_t find_box(const BoxDev* p, uint32_t n, uint64_t gi) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (p[mid].hist_begin <= gi) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int M, typename T, bool AGG>
__global__ void __launch_bounds__(256, 3) box_history_kernel(const BoxArgs a) {
  __shared__ mcd::Affine tab[64];
  // A single problem's record is read on every flight: keep it in shared memory.
  __shared__ __align__(16) unsigned char s_prob[sizeof(BoxDev)];
  // fp64, one problem: its mesh planes, read on every voxel crossing
  __shared__ double s_planes[sizeof(T) == 8 ? mcb::kMaxPlanes : 1];
  if (threadIdx.x == 0) {
    mcd::Affine sq{a.lcg.g, a.lcg.c};
    for (int j = 0; j < 64; ++j) { tab[j] = sq; sq = mcd::compose(sq, sq); }
  }
  if (a.nprob == 1) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(a.probs);
    uint64_t* dst = reinterpret_cast<uint64_t*>(s_prob);
    for (uint32_t i = threadIdx.x; i < sizeof(BoxDev) / 8; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const BoxDev* probs = a.nprob == 1 ? reinterpret_cast<const BoxDev*>(s_prob) : a.probs;
  const double* planes = nullptr;
  if (sizeof(T) == 8 && a.nprob == 1) {
    for (uint32_t j = threadIdx.x; j <= probs->mesh; j += blockDim.x) s_planes[j] = mcb::plane_of(*probs, (int)j);
    __syncthreads();
    planes = s_planes;
  }
  const unsigned kFull = 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  const mcd::Lcg l = a.lcg;

  uint64_t pool_next = 0, pool_end = 0;
  bool more = true, alive = false, primary = false;
  mcb::BoxCounts lc;
  lc.prob = -1;
  lc.clear();
  const BoxDev* P = probs;
  uint32_t pi = 0;
  mcs::Rng<M> r{0ull, 0ull};
  mcb::Part<T> q{};
  unsigned long long* base = nullptr;
  uint64_t gi = 0, events = 0, tbase = 0;

  for (;;) {
    unsigned dead = __ballot_sync(kFull, !alive);
    while (dead != 0u && more) {
      if (pool_next >= pool_end) {
        unsigned long long b0 = 0;
        if (lane == 0) b0 = atomicAdd(a.ticket, (unsigned long long)a.chunk);
        b0 = __shfl_sync(kFull, b0, 0);
        if (b0 >= a.total) { more = false; break; }
        pool_next = b0;
        pool_end = min((uint64_t)b0 + (uint64_t)a.chunk, (uint64_t)a.total);
      }
      const uint64_t avail = pool_end - pool_next;
      const unsigned rank = __popc(dead & lt_mask);
      if (!alive && rank < avail) {
        const uint64_t item = pool_next + rank;
        if (a.child_in == nullptr) {
          gi = a.range_begin + item;
          pi = a.nprob == 1 ? 0u : find_box(a.probs, a.nprob, gi);
          P = probs + pi;
          const uint64_t id = gi - P->hist_begin;
          const uint64_t nvox = (uint64_t)P->mesh * P->mesh * P->mesh;
          tbase = P->tally_offset + mcs::batch_of(id, P->n_hist, P->n_batches) * nvox;
          const uint64_t seed = P->seeding == MC_SEED_STRIDE
                                    ? mcs::skip_tab(tab, P->seed, P->stride_q * (P->id_offset + id)) & l.mask
                                    : mcd::hash_with(id, P->seed_hash) & l.mask;
          r = mcs::Rng<M>{seed, 0ull};
          mcb::box_source<M, T>(*P, r, l, q);
          primary = true;
        } else {
          const ChildRec c = a.child_in[item];
          pi = c.prob;
          P = probs + pi;
          tbase = c.tbase;
          r = mcs::Rng<M>{c.rng, 0ull};
          mcb::load_child<T>(c, q);
          primary = false;
        }
        if ((int)pi != lc.prob) { lc.flush(a.counts); lc.prob = (int)pi; }
        base = a.tally + tbase;
        events = 0;
        if (primary) ++lc.src;
        alive = true;
      }
      pool_next += min((uint64_t)__popc(dead), avail);
      dead = __ballot_sync(kFull, !alive);
    }
    if (__ballot_sync(kFull, alive) == 0u) break;
    if (!alive) continue;
    bool end = false;
    if (events == a.event_cap) {
      ++lc.capped;
      end = true;
    } else {
      ++events;
      ++lc.flights;
      const int o = mcb::box_flight<M, T>(*P, r, l, q, base, planes, AGG);
      if (o == mcb::kBoxLeak) {
        ++lc.leaks;
        end = true;
      } else if (o == mcb::kBoxCollide) {
        ++lc.coll;
        const int c = mcb::box_collide<M, T>(*P, r, l, q);
        if (c == mcb::kBoxKilled) {
          ++lc.kills;
          end = true;
        } else if (c >= mcb::kSplitBase + 2) {
          const uint32_t n = (uint32_t)(c - mcb::kSplitBase);
          ++lc.splits;
          lc.children += n - 1;
          for (uint32_t k = 0; k + 1 < n; ++k) {
            const unsigned long long idx = atomicAdd(a.child_out_count, 1ull);
            if (idx < a.child_cap) {
              mcb::store_child<T>(a.child_out[idx], q, mcb::child_seed(k, r.x, l.mask), pi, tbase);
            }
          }
        }
      }
    }
    if (end) {
      lc.draws += r.draws;
      if (r.draws > lc.maxd) lc.maxd = r.draws;
      if (primary) {
        if (P->stride_q != 0 && r.draws > P->stride_q) { ++lc.exh; lc.exd += r.draws - P->stride_q; }
        if (a.hist_state) a.hist_state[gi] = r.x & l.mask;
        if (a.hist_draws) a.hist_draws[gi] = r.draws;
      }
      alive = false;
      if (lc.draws > (1ull << 31)) lc.flush(a.counts);
    }
  }
  lc.flush_warp(a.counts);
}

}  // namespace

namespace {

template <int M, typename T, bool AGG>
int launch_box_gen(const BoxArgs& a, int block, int bps, int num_sms, cudaStream_t s) {
  auto k = box_history_kernel<M, T, AGG>;
  int per_sm = bps;
  if (per_sm <= 0) {
    int st = mci::cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, 0),
                              "cudaOccupancyMaxActiveBlocksPerMultiprocessor(box)");
    if (st != MC_OK) return st;
    if (per_sm < 1) per_sm = 1;
  }
  const uint64_t warps_needed = (a.total + a.chunk - 1) / a.chunk;
  const uint64_t blocks_needed = (warps_needed * 32 + block - 1) / block;
  const uint64_t full = (uint64_t)num_sms * (uint64_t)per_sm;
  const int grid = (int)std::max<uint64_t>(1, std::min(full, blocks_needed));
  k<<<grid, block, 0, s>>>(a);
  return mci::cuda_status(cudaGetLastError(), "box_history_kernel launch");
}

template <int M, typename T>
int run_box_history(const mci::BoxLaunch& L, cudaStream_t s) {
  BoxArgs a{};
  a.probs = static_cast<const BoxDev*>(L.d_probs);
  a.nprob = L.n_problems;
  a.chunk = L.chunk;
  a.tally = reinterpret_cast<unsigned long long*>(L.tally->d_bins);
  a.counts = reinterpret_cast<unsigned long long*>(L.tally->d_counts);
  a.hist_state = L.tally->d_hist_state;
  a.hist_draws = L.tally->d_hist_draws;
  a.lcg = mcd::Lcg{L.lcg.g, L.lcg.c, mcd::mask_of(L.lcg.m), L.lcg.m};
  a.event_cap = L.event_cap;
  a.ticket = L.d_ticket;
  a.child_cap = L.child_cap;
  ChildRec* bank[2] = {static_cast<ChildRec*>(L.d_child[0]), static_cast<ChildRec*>(L.d_child[1])};
  unsigned long long* cnt[2] = {L.d_child_count, L.d_child_count + 1};
  for (uint64_t start = 0; start < L.total; start += L.primary_chunk) {
    const uint64_t n = std::min<uint64_t>(L.primary_chunk, L.total - start);
    // generation 0: source histories
    MC_TRY_CUDA(cudaMemsetAsync(L.d_ticket, 0, sizeof(unsigned long long), s));
    MC_TRY_CUDA(cudaMemsetAsync(cnt[0], 0, sizeof(unsigned long long), s));
    a.child_in = nullptr;
    a.range_begin = L.range_begin + start;
    a.total = n;
    a.child_out = bank[0];
    a.child_out_count = cnt[0];
    int st = (L.tally_agg ? launch_box_gen<M, T, true> : launch_box_gen<M, T, false>)(a, L.block, L.blocks_per_sm, L.num_sms, s);
    if (st != MC_OK) return st;
    int cur = 0;
    for (int gen = 1;; ++gen) {
      unsigned long long made = 0;
      MC_TRY_CUDA(cudaMemcpyAsync(L.h_count, cnt[cur], sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      MC_TRY_CUDA(cudaStreamSynchronize(s));
      made = *L.h_count;
      if (made > L.child_cap) {
        mci::set_error("box transport: %llu children in one generation exceed the bank of %llu", made,
                       (unsigned long long)L.child_cap);
        return MC_ERR_CAPACITY;
      }
      if (made == 0) break;
      if ((uint32_t)gen > L.max_generations) {
        mci::set_error("box transport: more than %u generations of children", L.max_generations);
        return MC_ERR_TIMEOUT;
      }
      const int nxt = cur ^ 1;
      MC_TRY_CUDA(cudaMemsetAsync(L.d_ticket, 0, sizeof(unsigned long long), s));
      MC_TRY_CUDA(cudaMemsetAsync(cnt[nxt], 0, sizeof(unsigned long long), s));
      a.child_in = bank[cur];
      a.range_begin = 0;
      a.total = made;
      a.child_out = bank[nxt];
      a.child_out_count = cnt[nxt];
      st = (L.tally_agg ? launch_box_gen<M, T, true> : launch_box_gen<M, T, false>)(a, L.block, L.blocks_per_sm, L.num_sms, s);
      if (st != MC_OK) return st;
      cur = nxt;
    }
  }
  return MC_OK;
}

}  // namespace

namespace mci {

size_t box_dev_size() { return sizeof(BoxDev); }
size_t box_child_rec_size() { return sizeof(ChildRec); }

int box_fill_host(const mc_problem* src, uint32_t n, void* dst) {
  BoxDev* d = static_cast<BoxDev*>(dst);
  for (uint32_t i = 0; i < n; ++i) {
    const mc_box_spec* b = src[i].box;
    BoxDev q;
    std::memset(&q, 0, sizeof q);
    q.side = b->side;
    q.lo = b->inner_lo;
    q.hi = b->inner_hi;
    for (int r = 0; r < 2; ++r) {
      q.st[r] = b->sigma_t[r];
      q.c[r] = b->c[r];
      q.wl[r] = b->ww_low[r];
      q.wh[r] = b->ww_high[r];
      q.ws[r] = b->ww_survive[r];
      for (int g = 0; g < MC_BOX_MAX_GROUPS; ++g)
        for (int h = 0; h < MC_BOX_MAX_GROUPS; ++h) q.cdf[r][g][h] = b->scatter_cdf[r][g][h];
    }
    q.ng = b->n_groups;
    q.mesh = b->mesh;
    q.max_split = b->max_split;
    q.n_hist = src[i].n_histories;
    q.seed = src[i].seed;
    q.stride_q = src[i].stride_q;
    q.id_offset = src[i].id_offset;
    q.key = src[i].key;
    q.tally_offset = src[i].tally_offset;
    q.n_batches = src[i].n_batches;
    q.seeding = src[i].seeding;
    q.source = src[i].source;
    d[i] = q;
  }
  return MC_OK;
}

int box_prep(void* d_probs, uint32_t n, cudaStream_t s) {
  box_prep_kernel<<<1, 256, 0, s>>>(static_cast<BoxDev*>(d_probs), n);
  return cuda_status(cudaGetLastError(), "box_prep_kernel launch");
}

int box_history_run(const BoxLaunch& L, cudaStream_t s) {
  if (L.lcg.m == 63) return L.f32 ? run_box_history<63, float>(L, s) : run_box_history<63, double>(L, s);
  return L.f32 ? run_box_history<0, float>(L, s) : run_box_history<0, double>(L, s);
}

}  // namespace mci

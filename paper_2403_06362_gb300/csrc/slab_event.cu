// slab_event.cu -- the event-based slab schedule (Section 1 names the
// event-based algorithm of vector machines as the change of basis that
// reproducible seeding must survive).
//
// Particles live in a bank in device memory (structure of arrays) instead of
// registers.  Each iteration runs one kernel per event type over a queue of
// bank slots:
//   plan     (1 thread)  how many free slots to refill from the ticket
//   refill   new histories: seed (hash or stride), sample the source, queue
//            for flight
//   flight   one flight per queued particle: tally the track; leaks finish,
//            collisions are queued for the collision kernel
//   collide  absorption finishes the history, scattering re-queues it
//   advance  (1 thread)  swap the flight queues, test for completion
// The per-particle arithmetic is slab.cuh's slab_source, slab_flight and
// slab_collide -- the very functions the history kernel calls -- so every
// int64 tally contribution is the same and the totals are bit-identical to
// the history schedule.  The host launches iterations in batches (optionally
// as one captured CUDA graph per batch) and reads the completion flag between
// batches; no kernel waits on another.
//
// Once every history has started and the live particles no longer fill the
// GPU (at most tail_threshold), an iteration moves too few particles to pay
// for its five launches, and the longest chain would set the iteration
// count.  The advance kernel then flags the switch, and one tail kernel runs
// each live particle to its end from the bank, with the same slab_flight and
// slab_collide: the same draws and the same integer contributions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "slab.cuh"
#include "transport.h"

namespace {

using mcs::SlabDev;

struct EvCtl {
  unsigned int nfq[2];   // flight queue lengths
  unsigned int ncq;      // collision queue length
  unsigned int nfree;    // free-slot stack depth
  unsigned int cur;      // which flight queue is current
  unsigned int refill_n, refill_free_base;
  unsigned int done;
  unsigned long long refill_ticket_base;
  unsigned long long ticket;  // next history (relative to range_begin)
  unsigned long long iters;
};

struct EvBank {
  EvCtl* ctl;
  mcd::Affine* tab;  // maps of 2^j LCG steps (stride seeding)
  uint64_t *rng, *draws, *events, *gi, *coll, *scat, *tbase;
  double *x, *mu, *w;
  float *xf, *muf, *wf;
  uint32_t *prob, *fq0, *fq1, *cq, *freeq;
  uint32_t cap;
};

struct EvArgs {
  uint32_t tail_threshold;  // live particles at or below which the tail kernel takes over
  const SlabDev* probs;
  uint32_t nprob;
  uint64_t range_begin, total;
  unsigned long long* tally;
  unsigned long long* counts;
  uint64_t* hist_state;
  uint64_t* hist_draws;
  mcd::Lcg lcg;
  uint64_t event_cap;
  EvBank b;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Carves the bank arrays out of one buffer; returns the bytes needed.
size_t carve(void* base, uint32_t cap, EvBank* b) {
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  EvBank t{};
  t.ctl = reinterpret_cast<EvCtl*>(take(sizeof(EvCtl)));
  t.tab = reinterpret_cast<mcd::Affine*>(take(64 * sizeof(mcd::Affine)));
  t.rng = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  t.draws = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  t.events = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  t.gi = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  t.coll = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  t.scat = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  t.tbase = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  t.x = reinterpret_cast<double*>(take((size_t)cap * 8));
  t.mu = reinterpret_cast<double*>(take((size_t)cap * 8));
  t.w = reinterpret_cast<double*>(take((size_t)cap * 8));
  t.xf = reinterpret_cast<float*>(take((size_t)cap * 4));
  t.muf = reinterpret_cast<float*>(take((size_t)cap * 4));
  t.wf = reinterpret_cast<float*>(take((size_t)cap * 4));
  t.prob = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
  t.fq0 = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
  t.fq1 = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
  t.cq = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
  t.freeq = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
  t.cap = cap;
  if (b) *b = t;
  return off;
}

// Appends `slot` to a queue with one atomic per warp (all active lanes that
// call it append).
__device__ __forceinline__ void warp_append(unsigned int* counter, uint32_t* q, uint32_t slot) {
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned rank = __popc(mask & ((1u << lane) - 1u));
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  q[base + rank] = slot;
}

__device__ __forceinline__ uint32_t find_problem_ev(const SlabDev* p, uint32_t n, uint64_t gi) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (p[mid].hist_begin <= gi) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void ev_init_kernel(EvArgs a) {
  const EvBank& b = a.b;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < b.cap; i += nt) b.freeq[i] = (uint32_t)(b.cap - 1 - i);
  if (tid == 0) {
    EvCtl* c = b.ctl;
    c->nfq[0] = c->nfq[1] = 0;
    c->ncq = 0;
    c->nfree = b.cap;
    c->cur = 0;
    c->refill_n = c->refill_free_base = 0;
    c->done = a.total == 0 ? 1u : 0u;
    c->refill_ticket_base = 0;
    c->ticket = 0;
    c->iters = 0;
    mcd::Affine sq{a.lcg.g, a.lcg.c};
    for (int j = 0; j < 64; ++j) {
      b.tab[j] = sq;
      sq = mcd::compose(sq, sq);
    }
  }
}

__global__ void ev_plan_kernel(EvArgs a) {
  EvCtl* c = a.b.ctl;
  const uint64_t F = c->nfree, R = a.total - c->ticket;
  const uint64_t n = F < R ? F : R;
  c->refill_n = (unsigned int)n;
  c->refill_free_base = (unsigned int)(F - n);
  c->refill_ticket_base = c->ticket;
  c->nfree = (unsigned int)(F - n);
  c->ticket += n;
}

template <int M, bool F32>
__global__ void __launch_bounds__(256) ev_refill_kernel(EvArgs a) {
  const EvBank& b = a.b;
  const EvCtl* c = b.ctl;
  const uint32_t n = c->refill_n, fb = c->refill_free_base;
  const uint64_t tb = c->refill_ticket_base;
  uint32_t* fq = c->cur ? b.fq1 : b.fq0;
  unsigned int* nfq = &b.ctl->nfq[c->cur];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t slot = b.freeq[fb + t];
    const uint64_t gi = a.range_begin + tb + t;
    const uint32_t pi = a.nprob == 1 ? 0u : find_problem_ev(a.probs, a.nprob, gi);
    const SlabDev& P = a.probs[pi];
    const uint64_t id = gi - P.hist_begin;
    mcs::Rng<M> r{mcs::slab_seed(P, id, b.tab, a.lcg.mask), 0ull};
    mcs::SlabParticle q{};
    mcs::slab_source<M, F32>(P, r, a.lcg, q);
    b.rng[slot] = r.x;
    b.draws[slot] = r.draws;
    b.events[slot] = 0;
    b.gi[slot] = gi;
    b.coll[slot] = 0;
    b.scat[slot] = 0;
    b.tbase[slot] = P.tally_offset + mcs::batch_of(id, P.n_hist, P.n_batches) * P.n_bins;
    b.prob[slot] = pi;
    if constexpr (F32) {
      b.xf[slot] = q.xf; b.muf[slot] = q.muf; b.wf[slot] = q.wf;
    } else {
      b.x[slot] = q.x; b.mu[slot] = q.mu; b.w[slot] = q.w_mu;
    }
    warp_append(nfq, fq, slot);
  }
}

// Ends the history in `slot`: counters (into the thread's `ec`, flushed by
// its warp at the end of the kernel or here when the problem changes),
// per-history outputs, free the slot.
__device__ void ev_finish(const EvArgs& a, uint32_t slot, int outcome, uint64_t rng_x, uint64_t draws,
                          mcs::LaneCounts& ec) {
  const EvBank& b = a.b;
  const uint32_t pi = b.prob[slot];
  const SlabDev& P = a.probs[pi];
  if ((int)pi != ec.prob) { ec.flush(a.counts); ec.prob = (int)pi; }
  ++ec.src;
  ec.flights += (uint32_t)b.events[slot];
  ec.coll += (uint32_t)b.coll[slot];
  ec.scat += (uint32_t)b.scat[slot];
  if (outcome == mcs::kAbsorbed) ++ec.absn;
  else if (outcome == mcs::kLeakLo) ++ec.llo;
  else if (outcome == mcs::kLeakHi) ++ec.lhi;
  else ++ec.capped;
  ec.draws += draws;
  if (draws > ec.maxd) ec.maxd = draws;
  if (P.stride_q != 0 && draws > P.stride_q) {
    ++ec.exh;
    ec.exd += draws - P.stride_q;
  }
  const uint64_t gi = b.gi[slot];
  if (a.hist_state) a.hist_state[gi] = rng_x & a.lcg.mask;
  if (a.hist_draws) a.hist_draws[gi] = draws;
  if (ec.draws > (1ull << 31) || ec.flights > (1u << 30)) ec.flush(a.counts);
  const unsigned int k = atomicAdd(&b.ctl->nfree, 1u);
  b.freeq[k] = slot;
}

template <int M, bool F32>
__global__ void __launch_bounds__(256) ev_flight_kernel(EvArgs a) {
  const EvBank& b = a.b;
  const unsigned int cur = b.ctl->cur;
  const uint32_t n = b.ctl->nfq[cur];
  const uint32_t* fq = cur ? b.fq1 : b.fq0;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  mcs::LaneCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t slot = fq[t];
    const SlabDev& P = a.probs[b.prob[slot]];
    mcs::Rng<M> r{b.rng[slot], b.draws[slot]};
    const uint64_t ev = b.events[slot];
    if (ev == a.event_cap) {
      ev_finish(a, slot, -1, r.x, r.draws, ec);
      continue;
    }
    b.events[slot] = ev + 1;
    mcs::SlabParticle q{};
    if constexpr (F32) {
      q.xf = b.xf[slot]; q.muf = b.muf[slot]; q.wf = b.wf[slot];
    } else {
      q.x = b.x[slot]; q.mu = b.mu[slot]; q.w_mu = b.w[slot];
    }
    const mcs::Sink sink{a.tally + b.tbase[slot], nullptr, nullptr, false};
    const int o = mcs::slab_flight<M, F32>(P, r, a.lcg, q, sink);
    if (o != mcs::kCollide) {
      ev_finish(a, slot, o, r.x, r.draws, ec);
      continue;
    }
    b.rng[slot] = r.x;
    b.draws[slot] = r.draws;
    if constexpr (F32) b.xf[slot] = q.xf; else b.x[slot] = q.x;
    warp_append(&b.ctl->ncq, b.cq, slot);
  }
  ec.flush_warp(a.counts);
}

template <int M, bool F32>
__global__ void __launch_bounds__(256) ev_collide_kernel(EvArgs a) {
  const EvBank& b = a.b;
  const unsigned int nxt = b.ctl->cur ^ 1u;
  const uint32_t n = b.ctl->ncq;
  uint32_t* fq = nxt ? b.fq1 : b.fq0;
  unsigned int* nfq = &b.ctl->nfq[nxt];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  mcs::LaneCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t slot = b.cq[t];
    const SlabDev& P = a.probs[b.prob[slot]];
    mcs::Rng<M> r{b.rng[slot], b.draws[slot]};
    mcs::SlabParticle q{};
    if constexpr (F32) {
      q.xf = b.xf[slot]; q.muf = b.muf[slot]; q.wf = b.wf[slot];
    } else {
      q.x = b.x[slot]; q.mu = b.mu[slot]; q.w_mu = b.w[slot];
    }
    b.coll[slot] += 1;
    const int o = mcs::slab_collide<M, F32>(P, r, a.lcg, q);
    if (o == mcs::kAbsorbed) {
      ev_finish(a, slot, o, r.x, r.draws, ec);
      continue;
    }
    b.scat[slot] += 1;
    b.rng[slot] = r.x;
    b.draws[slot] = r.draws;
    if constexpr (F32) {
      b.muf[slot] = q.muf; b.wf[slot] = q.wf;
    } else {
      b.mu[slot] = q.mu; b.w[slot] = q.w_mu;
    }
    warp_append(nfq, fq, slot);
  }
  ec.flush_warp(a.counts);
}

__global__ void ev_advance_kernel(EvArgs a) {
  EvCtl* c = a.b.ctl;
  const unsigned int cur = c->cur;
  c->nfq[cur] = 0;
  c->ncq = 0;
  c->cur = cur ^ 1u;
  const unsigned int live = c->nfq[cur ^ 1u];
  // 1: finished; 2: every history started and few enough live for the tail kernel
  c->done = c->ticket < a.total ? 0u : (live == 0 ? 1u : (live <= a.tail_threshold ? 2u : 0u));
  c->iters += 1;
}

// The tail: each live particle of the current flight queue flies and
// collides to the end of its history in one thread.
template <int M, bool F32>
__global__ void __launch_bounds__(256) ev_tail_kernel(EvArgs a) {
  const EvBank& b = a.b;
  const unsigned int cur = b.ctl->cur;
  const uint32_t n = b.ctl->nfq[cur];
  const uint32_t* fq = cur ? b.fq1 : b.fq0;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  mcs::LaneCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t slot = fq[t];
    const SlabDev& P = a.probs[b.prob[slot]];
    mcs::Rng<M> r{b.rng[slot], b.draws[slot]};
    uint64_t ev = b.events[slot];
    uint32_t co = 0, sc = 0;
    mcs::SlabParticle q{};
    if constexpr (F32) {
      q.xf = b.xf[slot]; q.muf = b.muf[slot]; q.wf = b.wf[slot];
    } else {
      q.x = b.x[slot]; q.mu = b.mu[slot]; q.w_mu = b.w[slot];
    }
    const mcs::Sink sink{a.tally + b.tbase[slot], nullptr, nullptr, false};
    int outcome;
    for (;;) {
      if (ev == a.event_cap) { outcome = -1; break; }
      ++ev;
      outcome = mcs::slab_event<M, F32>(P, r, a.lcg, q, sink, co, sc);
      if (outcome != mcs::kContinue) break;
    }
    b.events[slot] = ev;
    b.coll[slot] += co;
    b.scat[slot] += sc;
    ev_finish(a, slot, outcome, r.x, r.draws, ec);
  }
  ec.flush_warp(a.counts);
}

constexpr int kIterPerBatch = 32;

template <int M, bool F32>
void enqueue_batch(const EvArgs& a, int grid, cudaStream_t s) {
  for (int k = 0; k < kIterPerBatch; ++k) {
    ev_plan_kernel<<<1, 1, 0, s>>>(a);
    ev_refill_kernel<M, F32><<<grid, 256, 0, s>>>(a);
    ev_flight_kernel<M, F32><<<grid, 256, 0, s>>>(a);
    ev_collide_kernel<M, F32><<<grid, 256, 0, s>>>(a);
    ev_advance_kernel<<<1, 1, 0, s>>>(a);
  }
}

template <int M, bool F32>
int run_event(const EvArgs& a, int grid, cudaStream_t capture_stream, unsigned int* h_done, uint64_t max_batches,
              cudaStream_t s) {
  ev_init_kernel<<<grid, 256, 0, s>>>(a);
  MC_TRY_CUDA(cudaGetLastError());
  cudaGraphExec_t exec = nullptr;
  if (capture_stream) {
    cudaGraph_t g = nullptr;
    MC_TRY_CUDA(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_batch<M, F32>(a, grid, capture_stream);
    cudaError_t e = cudaStreamEndCapture(capture_stream, &g);
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaStreamEndCapture(event batch)");
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaGraphInstantiate(event batch)");
  }
  int st = MC_OK;
  for (uint64_t batch = 0;; ++batch) {
    if (batch == max_batches) {
      mci::set_error("event schedule: %llu iterations without completing", (unsigned long long)(batch * kIterPerBatch));
      st = MC_ERR_TIMEOUT;
      break;
    }
    if (exec) {
      cudaError_t e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) { st = mci::cuda_status(e, "cudaGraphLaunch(event batch)"); break; }
    } else {
      enqueue_batch<M, F32>(a, grid, s);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) { st = mci::cuda_status(e, "event kernels launch"); break; }
    }
    cudaError_t e = cudaMemcpyAsync(h_done, &a.b.ctl->done, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = mci::cuda_status(e, "event schedule completion check"); break; }
    if (*h_done == 2u) {  // the rest of the histories in one kernel
      ev_tail_kernel<M, F32><<<grid, 256, 0, s>>>(a);
      st = mci::cuda_status(cudaGetLastError(), "ev_tail_kernel launch");
      break;
    }
    if (*h_done) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  return st;
}

}  // namespace

namespace mci {

size_t slab_bank_bytes(uint32_t cap) { return carve(nullptr, cap, nullptr); }

int slab_event_run(const SlabLaunch& L, void* d_bank, uint32_t cap, unsigned int* h_done,
                   cudaStream_t capture_stream, cudaStream_t s) {
  EvArgs a{};
  a.probs = static_cast<const SlabDev*>(L.d_probs);
  a.nprob = L.n_problems;
  a.range_begin = L.range_begin;
  a.total = L.total;
  a.tally = reinterpret_cast<unsigned long long*>(L.tally->d_bins);
  a.counts = reinterpret_cast<unsigned long long*>(L.tally->d_counts);
  a.hist_state = L.tally->d_hist_state;
  a.hist_draws = L.tally->d_hist_draws;
  a.lcg = mcd::Lcg{L.lcg.g, L.lcg.c, mcd::mask_of(L.lcg.m), L.lcg.m};
  a.event_cap = L.event_cap;
  carve(d_bank, cap, &a.b);
  const int grid = std::max(1, L.num_sms * 4);
  a.tail_threshold = (uint32_t)L.num_sms * 1024u;
  // Every iteration flies each live particle once, so the longest history
  // bounds the iteration count; the cap below is a safety net only.
  const uint64_t max_iters = std::min<uint64_t>(L.event_cap, 1ull << 36) * 2 + (L.total / cap + 2) * 4 + 64;
  uint64_t max_batches = max_iters / kIterPerBatch + 2;
  if (L.event_iterations != ~0ull)  // a caller's bound (mc_limits), in whole batches
    max_batches = L.event_iterations / kIterPerBatch + (L.event_iterations % kIterPerBatch != 0);
  if (L.lcg.m == 63) {
    return L.f32 ? run_event<63, true>(a, grid, capture_stream, h_done, max_batches, s)
                 : run_event<63, false>(a, grid, capture_stream, h_done, max_batches, s);
  }
  return L.f32 ? run_event<0, true>(a, grid, capture_stream, h_done, max_batches, s)
               : run_event<0, false>(a, grid, capture_stream, h_done, max_batches, s);
}

}  // namespace mci

// slab_event.cu -- the event-based slab schedule (Section 1 names the
// event-based algorithm of vector machines as the change of basis that
// reproducible seeding must survive).
//
// Particles live in device banks instead of registers, one array per field
// (structure of arrays).  Each iteration is ONE kernel that streams the
// current bank in slot order -- every field load of a warp is one coalesced
// access -- and moves each particle one step: it flies (tallying its track)
// and, if it stops at a collision site, collides.  Survivors are appended to
// the other bank (one atomic per group of converged lanes, so a group's
// stores land in consecutive slots), which keeps the bank dense: no dead
// slots, no queue.  A history that ended is replaced in the same pass by
// the next history from a ticket (its seed and source sample), so the bank
// stays full while histories remain.  The block that finishes last (a
// counter, no waiting) swaps the banks and sets the completion flag.  The
// host launches iterations in batches (optionally one captured CUDA graph
// per batch) and reads the flag between batches; no kernel waits on another.
//
// The per-particle arithmetic is slab.cuh's slab_source, slab_flight and
// slab_collide -- the very functions the history kernel calls -- so every
// int64 tally contribution is the same and the totals are bit-identical to
// the history schedule.  Once every history has started and the live
// particles no longer fill the GPU (at most tail_threshold), one tail kernel
// runs each live particle to its end from the bank.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "internal.h"
#include "slab.cuh"
#include "transport.h"

namespace {

using mcs::SlabDev;

struct EvCtl {
  unsigned int n[2];         // particles in each bank
  unsigned int cur;          // the bank the next iteration reads
  unsigned int done;         // 1: finished; 2: the tail kernel next
  unsigned int blocks_done;  // blocks of the running iteration that finished
  unsigned int pad;
  unsigned long long ticket;  // next history (relative to range_begin)
  unsigned long long iters;
};

// One bank: an array per field -- the fp64 path's x, mu and 2^32/|mu|, or the
// fp32 path's xf, muf and 1/|muf|, then the stream, its draw and flight
// counts, the history index, the tally row, the problem and, in launches of
// several problems, the history's collision and scattering counts so far
// (68 + 16 bytes fp64, 60 + 16 fp32 per particle).  There a history's counters
// are added to its problem's when it ends, so a pass touches the counters
// once per ended history, not once per event; a single problem's lanes count
// every event in registers.
template <bool F32>
struct EvSoA {
  using P = typename std::conditional<F32, float, double>::type;
  P *x, *mu, *w;
  float* xlo;  // fp32 path: the low part of the position
  uint64_t *rng, *draws, *events, *gi, *tbase;
  uint32_t* prob;
  uint64_t *coll, *scat;
};

template <bool F32>
struct EvBank {
  EvCtl* ctl;
  mcd::Affine* tab;  // maps of 2^j LCG steps (stride seeding)
  EvSoA<F32> f[2];
  uint32_t cap;
};

template <bool F32>
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
  uint32_t smem_edges;    // one problem: its n_bins + 1 edges and n_bins widths in shared memory (0: none)
  const double* tables;   // else each problem's edge and width tables in global memory (nullable)
  uint32_t smem_counts;   // 1: 2..kSmemCountProblems problems, counters staged in shared memory
  mcs::Order order;       // processing order of several problems (empty: id order)
  EvBank<F32> b;
};

// Launches of at most this many problems stage their counters per block in
// shared memory (a lane's counters go there when its history's problem
// differs from the last one's, and the block adds them to the problems'
// counters once per pass).
constexpr uint32_t kSmemCountProblems = 256;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

template <bool F32>
size_t carve(void* base, uint32_t cap, EvBank<F32>* b) {
  using P = typename EvSoA<F32>::P;
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  EvBank<F32> t{};
  t.ctl = reinterpret_cast<EvCtl*>(take(sizeof(EvCtl)));
  t.tab = reinterpret_cast<mcd::Affine*>(take(64 * sizeof(mcd::Affine)));
  for (int k = 0; k < 2; ++k) {
    EvSoA<F32>& f = t.f[k];
    f.x = reinterpret_cast<P*>(take((size_t)cap * sizeof(P)));
    f.mu = reinterpret_cast<P*>(take((size_t)cap * sizeof(P)));
    f.w = reinterpret_cast<P*>(take((size_t)cap * sizeof(P)));
    f.xlo = F32 ? reinterpret_cast<float*>(take((size_t)cap * 4)) : nullptr;
    uint64_t** uu[] = {&f.rng, &f.draws, &f.events, &f.gi, &f.tbase};
    for (uint64_t** u : uu) *u = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
    f.prob = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
    f.coll = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
    f.scat = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  }
  t.cap = cap;
  if (b) *b = t;
  return off;
}

// A particle as the kernels hold it.
struct EvLive {
  mcs::SlabParticle q;
  uint64_t rng, draws, events, gi, tbase, coll, scat;
  uint32_t prob;
};

template <bool F32>
__device__ __forceinline__ void load_live(const EvSoA<F32>& f, uint32_t s, EvLive& v, bool per_hist) {
  v.q = mcs::SlabParticle{};
  if constexpr (F32) {
    v.q.xf = f.x[s]; v.q.xlo = f.xlo[s]; v.q.muf = f.mu[s]; v.q.wf = f.w[s];
  } else {
    v.q.x = f.x[s]; v.q.mu = f.mu[s]; v.q.w_mu = f.w[s];
  }
  v.rng = f.rng[s];
  v.draws = f.draws[s];
  v.events = f.events[s];
  v.gi = f.gi[s];
  v.tbase = f.tbase[s];
  v.prob = f.prob[s];
  v.coll = per_hist ? f.coll[s] : 0ull;
  v.scat = per_hist ? f.scat[s] : 0ull;
}

template <bool F32>
__device__ __forceinline__ void store_live(const EvSoA<F32>& f, uint32_t s, const EvLive& v, bool per_hist) {
  if constexpr (F32) {
    f.x[s] = v.q.xf; f.xlo[s] = v.q.xlo; f.mu[s] = v.q.muf; f.w[s] = v.q.wf;
  } else {
    f.x[s] = v.q.x; f.mu[s] = v.q.mu; f.w[s] = v.q.w_mu;
  }
  f.rng[s] = v.rng;
  f.draws[s] = v.draws;
  f.events[s] = v.events;
  f.gi[s] = v.gi;
  f.tbase[s] = v.tbase;
  f.prob[s] = v.prob;
  if (per_hist) {
    f.coll[s] = v.coll;
    f.scat[s] = v.scat;
  }
}

// A slot in a bank for each converged lane that asks (one atomic per
// group: the group's slots are consecutive).
__device__ __forceinline__ uint32_t take_slot(unsigned int* counter) {
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned rank = __popc(mask & ((1u << lane) - 1u));
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(counter, (unsigned)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + rank;
}

// The next history for each converged lane that asks (one atomic per
// group); a value >= total once the ticket has run out.
__device__ __forceinline__ unsigned long long take_history(unsigned long long* ticket) {
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned rank = __popc(mask & ((1u << lane) - 1u));
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(ticket, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + rank;
}

// Starts the history at ticket position t in `v`.
template <int M, bool F32>
__device__ __forceinline__ void start_history(const EvArgs<F32>& a, const mcd::Affine* tab, uint64_t t, EvLive& v) {
  uint32_t pi;
  uint64_t gi;
  mcs::ticket_history(a.probs, a.nprob, a.range_begin, a.order, t, pi, gi);
  const SlabDev& P = a.probs[pi];
  const uint64_t id = gi - P.hist_begin;
  mcs::Rng<M> r{mcs::slab_seed(P, id, tab, a.lcg.mask), 0ull};
  v.q = mcs::SlabParticle{};
  mcs::slab_source<M, F32>(P, r, a.lcg, v.q);
  v.prob = pi;
  v.rng = r.x;
  v.draws = r.draws;
  v.events = 0;
  v.coll = 0;
  v.scat = 0;
  v.gi = gi;
  v.tbase = P.tally_offset + mcs::batch_of(id, P.n_hist, P.n_batches) * P.n_bins;
}

// The end of a history: its counters into the thread's `ec` (flushed into
// `cnt` -- the block's shared-memory counters or the problems' own -- by its
// warp at the end of the kernel, or when the problem changes) and its
// per-history outputs.
template <bool F32>
__device__ void ev_finish(const EvArgs<F32>& a, const SlabDev& P, const EvLive& v, int outcome,
                          mcs::LaneCounts& ec, unsigned long long* cnt) {
  if ((int)v.prob != ec.prob) { ec.flush(cnt); ec.prob = (int)v.prob; }
  if (!a.smem_counts) {
    // one problem: flights, collisions and scatters were counted per event
  } else if (v.events < (1ull << 30)) {
    ec.flights += (uint32_t)v.events;
    ec.coll += (uint32_t)v.coll;
    ec.scat += (uint32_t)v.scat;
  } else {  // a history too long for the 32-bit lane counters
    unsigned long long* c = a.counts + (size_t)v.prob * MC_NCOUNT;
    atomicAdd(c + MC_C_FLIGHTS, (unsigned long long)v.events);
    atomicAdd(c + MC_C_COLLISIONS, (unsigned long long)v.coll);
    atomicAdd(c + MC_C_SCATTERS, (unsigned long long)v.scat);
  }
  ++ec.src;
  if (outcome == mcs::kAbsorbed) ++ec.absn;
  else if (outcome == mcs::kLeakLo) ++ec.llo;
  else if (outcome == mcs::kLeakHi) ++ec.lhi;
  else ++ec.capped;
  ec.draws += v.draws;
  if (v.draws > ec.maxd) ec.maxd = v.draws;
  if (P.stride_q != 0 && v.draws > P.stride_q) {
    ++ec.exh;
    ec.exd += v.draws - P.stride_q;
  }
  if (a.hist_state) a.hist_state[v.gi] = v.rng & a.lcg.mask;
  if (a.hist_draws) a.hist_draws[v.gi] = v.draws;
  if (ec.draws > (1ull << 31) || ec.flights > (1u << 30) || ec.coll > (1u << 30)) ec.flush(cnt);
}

// The block's counter staging: zeroed at the start of a pass (nullptr: the
// lanes flush into the problems' counters directly).
template <bool F32>
__device__ __forceinline__ unsigned long long* stage_counts(const EvArgs<F32>& a) {
  extern __shared__ unsigned long long s_cnt[];
  if (!a.smem_counts) return nullptr;
  for (uint32_t i = threadIdx.x; i < a.nprob * MC_NCOUNT; i += blockDim.x) s_cnt[i] = 0ull;
  __syncthreads();
  return s_cnt;
}

// Adds the block's staged counters to the problems' counters.
template <bool F32>
__device__ __forceinline__ void flush_counts(const EvArgs<F32>& a, const unsigned long long* s_cnt) {
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < a.nprob * MC_NCOUNT; i += blockDim.x) {
    const unsigned long long v = s_cnt[i];
    if (v == 0ull) continue;
    if (i % MC_NCOUNT == MC_C_MAX_DRAWS) atomicMax(a.counts + i, v);
    else atomicAdd(a.counts + i, v);
  }
}

// The tally sink of a particle: its batch row, and the bin edge and width
// tables (shared memory for one problem, else global, else none).
template <bool F32>
__device__ __forceinline__ mcs::Sink sink_of(const EvArgs<F32>& a, const SlabDev& P, const EvLive& v,
                                             const double* s_edges) {
  mcs::Sink s{a.tally + v.tbase, nullptr, nullptr, false};
  if (s_edges) {
    s.edges = s_edges;
    s.widths = s_edges + a.smem_edges;
  } else if (a.tables) {
    s.edges = a.tables + P.tab_off;
    s.widths = s.edges + P.n_bins + 1;
  }
  return s;
}

// One problem: its edges and widths into shared memory (the same fp64
// values the prep kernel writes to the global tables).
template <bool F32>
__device__ __forceinline__ const double* stage_edges(const EvArgs<F32>& a) {
  extern __shared__ double s_tab[];
  if (a.smem_edges == 0) return nullptr;
  const SlabDev& p0 = a.probs[0];
  for (uint32_t j = threadIdx.x; j < a.smem_edges; j += blockDim.x) s_tab[j] = mcs::slab_edge(p0, (int)j);
  for (uint32_t j = threadIdx.x; j + 1 < a.smem_edges; j += blockDim.x)
    s_tab[a.smem_edges + j] = __dsub_rn(mcs::slab_edge(p0, (int)j + 1), mcs::slab_edge(p0, (int)j));
  __syncthreads();
  return s_tab;
}

// First pass: histories 0..min(cap, total)-1 into bank 0, and the control
// block reset.
template <int M, bool F32>
__global__ void __launch_bounds__(256) ev_init_kernel(EvArgs<F32> a) {
  __shared__ mcd::Affine tab[64];
  if (threadIdx.x == 0) {
    mcd::Affine sq{a.lcg.g, a.lcg.c};
    for (int j = 0; j < 64; ++j) { tab[j] = sq; sq = mcd::compose(sq, sq); }
  }
  __syncthreads();
  const EvBank<F32>& b = a.b;
  const uint64_t n = a.total < b.cap ? a.total : b.cap;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += nt) {
    EvLive v;
    start_history<M, F32>(a, tab, i, v);
    store_live<F32>(b.f[0], (uint32_t)i, v, a.smem_counts != 0u);
  }
  if (tid == 0) {
    EvCtl* c = b.ctl;
    c->n[0] = (unsigned int)n;
    c->n[1] = 0;
    c->cur = 0;
    // a generation that starts with every item in the bank and no more live
    // particles than the tail threshold goes straight to the tail kernel
    c->done = n == 0 ? 1u : ((n == a.total && n <= a.tail_threshold) ? 2u : 0u);
    c->blocks_done = 0;
    c->pad = 0;
    c->ticket = n;
    c->iters = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x < 64) b.tab[threadIdx.x] = tab[threadIdx.x];
}

// One iteration: each particle of the current bank flies once and, at a
// collision site, collides; survivors, and the histories that replace ended
// ones, go to the other bank.  The last block to finish advances the
// control block.
template <int M, bool F32>
__global__ void __launch_bounds__(256) ev_step_kernel(EvArgs<F32> a) {
  const double* s_edges = stage_edges<F32>(a);
  unsigned long long* const s_cnt = stage_counts<F32>(a);
  unsigned long long* const cnt = s_cnt ? s_cnt : a.counts;
  const bool per_hist = a.smem_counts != 0u;  // counts carried per history (several problems)
  const EvBank<F32>& b = a.b;
  EvCtl* c = b.ctl;
  const unsigned int cur = c->cur;
  const uint32_t n = c->n[cur];
  const EvSoA<F32>& fin = b.f[cur];
  const EvSoA<F32>& fout = b.f[cur ^ 1u];
  unsigned int* nout = &c->n[cur ^ 1u];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  mcs::LaneCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    EvLive v;
    load_live<F32>(fin, (uint32_t)t, v, per_hist);
    const SlabDev& P = a.probs[v.prob];
    mcs::Rng<M> r{v.rng, v.draws};
    int outcome = mcs::kContinue;
    if (v.events == a.event_cap) {
      outcome = -1;
    } else {
      ++v.events;
      if (!per_hist) {
        if ((int)v.prob != ec.prob) { ec.flush(cnt); ec.prob = (int)v.prob; }
        ++ec.flights;
      }
      outcome = mcs::slab_flight<M, F32>(P, r, a.lcg, v.q, sink_of<F32>(a, P, v, s_edges));
      if (outcome == mcs::kCollide) {
        ++v.coll;
        outcome = mcs::slab_collide<M, F32>(P, r, a.lcg, v.q);
        if (outcome == mcs::kContinue) ++v.scat;
        if (!per_hist) {
          ++ec.coll;
          if (outcome == mcs::kContinue) ++ec.scat;
        }
      }
    }
    v.rng = r.x;
    v.draws = r.draws;
    bool keep = true;
    if (outcome != mcs::kContinue) {
      ev_finish<F32>(a, P, v, outcome, ec, cnt);
      const unsigned long long h = take_history(&c->ticket);
      if (h < a.total) start_history<M, F32>(a, b.tab, h, v);
      else keep = false;
    }
    if (keep) store_live<F32>(fout, take_slot(nout), v, per_hist);
  }
  ec.flush_warp(cnt);
  if (s_cnt) flush_counts<F32>(a, s_cnt);
  // The last block to finish advances: the other blocks' stores and slot
  // counts are visible after their fence and counter increment.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(&c->blocks_done, 1u);
    if (prev == gridDim.x - 1u) {
      __threadfence();
      const unsigned int live = atomicAdd(nout, 0u);
      const unsigned long long tk = atomicAdd(&c->ticket, 0ull);
      c->n[cur] = 0u;
      c->cur = cur ^ 1u;
      c->blocks_done = 0u;
      c->iters += 1;
      c->done = tk < a.total ? 0u : (live == 0 ? 1u : (live <= a.tail_threshold ? 2u : 0u));
      __threadfence();
    }
  }
}

// The tail: each particle of the current bank flies and collides to the end
// of its history in one thread.
template <int M, bool F32>
__global__ void __launch_bounds__(256) ev_tail_kernel(EvArgs<F32> a) {
  const double* s_edges = stage_edges<F32>(a);
  unsigned long long* const s_cnt = stage_counts<F32>(a);
  unsigned long long* const cnt = s_cnt ? s_cnt : a.counts;
  const EvBank<F32>& b = a.b;
  const unsigned int cur = b.ctl->cur;
  const uint32_t n = b.ctl->n[cur];
  const EvSoA<F32>& fin = b.f[cur];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  mcs::LaneCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    EvLive v;
    load_live<F32>(fin, (uint32_t)t, v, a.smem_counts != 0u);
    const SlabDev& P = a.probs[v.prob];
    mcs::Rng<M> r{v.rng, v.draws};
    const mcs::Sink sink = sink_of<F32>(a, P, v, s_edges);
    const uint64_t ev0 = v.events, co0 = v.coll, sc0 = v.scat;
    int outcome;
    for (;;) {
      if (v.events == a.event_cap) { outcome = -1; break; }
      ++v.events;
      outcome = mcs::slab_flight<M, F32>(P, r, a.lcg, v.q, sink);
      if (outcome != mcs::kCollide) break;
      ++v.coll;
      outcome = mcs::slab_collide<M, F32>(P, r, a.lcg, v.q);
      if (outcome != mcs::kContinue) break;
      ++v.scat;
    }
    if (!a.smem_counts) {  // one problem: this kernel's events into the lane counters
      if ((int)v.prob != ec.prob) { ec.flush(cnt); ec.prob = (int)v.prob; }
      const uint64_t fl = v.events - ev0;
      if (fl < (1ull << 30)) {
        ec.flights += (uint32_t)fl;
        ec.coll += (uint32_t)(v.coll - co0);
        ec.scat += (uint32_t)(v.scat - sc0);
        if (ec.flights > (1u << 30)) ec.flush(cnt);
      } else {  // a history too long for the 32-bit lane counters
        unsigned long long* c = a.counts + (size_t)v.prob * MC_NCOUNT;
        atomicAdd(c + MC_C_FLIGHTS, (unsigned long long)fl);
        atomicAdd(c + MC_C_COLLISIONS, (unsigned long long)(v.coll - co0));
        atomicAdd(c + MC_C_SCATTERS, (unsigned long long)(v.scat - sc0));
      }
    }
    v.rng = r.x;
    v.draws = r.draws;
    ev_finish<F32>(a, P, v, outcome, ec, cnt);
  }
  ec.flush_warp(cnt);
  if (s_cnt) flush_counts<F32>(a, s_cnt);
}

constexpr int kIterPerBatch = 32;

template <int M, bool F32>
void enqueue_batch(const EvArgs<F32>& a, int grid, size_t smem, cudaStream_t s) {
  for (int k = 0; k < kIterPerBatch; ++k) ev_step_kernel<M, F32><<<grid, 256, smem, s>>>(a);
}

template <int M, bool F32>
int run_event(const EvArgs<F32>& a, int grid, size_t smem, cudaStream_t capture_stream, unsigned int* h_done,
              uint64_t max_batches, cudaStream_t s) {
  ev_init_kernel<M, F32><<<grid, 256, 0, s>>>(a);
  MC_TRY_CUDA(cudaGetLastError());
  cudaGraphExec_t exec = nullptr;
  if (capture_stream) {
    cudaGraph_t g = nullptr;
    MC_TRY_CUDA(cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_batch<M, F32>(a, grid, smem, capture_stream);
    cudaError_t e = cudaStreamEndCapture(capture_stream, &g);
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaStreamEndCapture(event batch)");
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaGraphInstantiate(event batch)");
  }
  int st = MC_OK;
  for (uint64_t batch = 0;; ++batch) {
    // the completion flag as the init kernel or the last iteration left it
    cudaError_t e = cudaMemcpyAsync(h_done, &a.b.ctl->done, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = mci::cuda_status(e, "event schedule completion check"); break; }
    if (*h_done == 2u) {  // the rest of the histories in one kernel
      ev_tail_kernel<M, F32><<<grid, 256, smem, s>>>(a);
      st = mci::cuda_status(cudaGetLastError(), "ev_tail_kernel launch");
      break;
    }
    if (*h_done) break;
    if (batch == max_batches) {
      mci::set_error("event schedule: %llu iterations without completing", (unsigned long long)(batch * kIterPerBatch));
      st = MC_ERR_TIMEOUT;
      break;
    }
    if (exec) {
      e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) { st = mci::cuda_status(e, "cudaGraphLaunch(event batch)"); break; }
    } else {
      enqueue_batch<M, F32>(a, grid, smem, s);
      e = cudaGetLastError();
      if (e != cudaSuccess) { st = mci::cuda_status(e, "event kernels launch"); break; }
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  return st;
}

template <int M, bool F32>
int slab_event_run_t(const mci::SlabLaunch& L, void* d_bank, uint32_t cap, unsigned int* h_done,
                     cudaStream_t capture_stream, cudaStream_t s) {
  EvArgs<F32> a{};
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
  // One problem with at most 4095 bins: its edge and width tables in shared
  // memory; otherwise each problem's tables in global memory.
  a.smem_edges = (L.n_problems == 1 && L.single_n_bins + 1 <= 4096) ? L.single_n_bins + 1 : 0u;
  a.tables = a.smem_edges ? nullptr : static_cast<const double*>(L.d_tables);
  a.smem_counts = (L.n_problems > 1 && L.n_problems <= kSmemCountProblems) ? 1u : 0u;
  a.order = mcs::Order{L.d_order, L.d_order_begin};
  const size_t smem = a.smem_edges ? (size_t)a.smem_edges * 16u
                                   : (a.smem_counts ? (size_t)L.n_problems * MC_NCOUNT * 8u : 0u);
  carve<F32>(d_bank, cap, &a.b);
  // One wave of resident blocks: every block of an iteration runs at once.
  int per_sm = 0;
  MC_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ev_step_kernel<M, F32>, 256, smem));
  const int grid = std::max(1, L.num_sms * std::max(per_sm, 1));
  a.tail_threshold = (uint32_t)L.num_sms * 1024u;
  // Each iteration moves every live particle one flight and the bank refills
  // from the ticket; the bound below is a safety net only.
  const uint64_t max_iters = std::min<uint64_t>(L.event_cap, 1ull << 36) * 2 + (L.total / cap + 2) * 4 + 64;
  uint64_t max_batches = max_iters / kIterPerBatch + 2;
  if (L.event_iterations != ~0ull)  // a caller's bound (mc_limits), in whole batches
    max_batches = L.event_iterations / kIterPerBatch + (L.event_iterations % kIterPerBatch != 0);
  return run_event<M, F32>(a, grid, smem, capture_stream, h_done, max_batches, s);
}

}  // namespace

namespace mci {

size_t slab_bank_bytes(uint32_t cap) {
  return std::max(carve<false>(nullptr, cap, nullptr), carve<true>(nullptr, cap, nullptr));
}

int slab_event_run(const SlabLaunch& L, void* d_bank, uint32_t cap, unsigned int* h_done,
                   cudaStream_t capture_stream, cudaStream_t s) {
  if (L.lcg.m == 63) {
    return L.f32 ? slab_event_run_t<63, true>(L, d_bank, cap, h_done, capture_stream, s)
                 : slab_event_run_t<63, false>(L, d_bank, cap, h_done, capture_stream, s);
  }
  return L.f32 ? slab_event_run_t<0, true>(L, d_bank, cap, h_done, capture_stream, s)
               : slab_event_run_t<0, false>(L, d_bank, cap, h_done, capture_stream, s);
}

}  // namespace mci

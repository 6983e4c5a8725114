// box_event.cu -- event-based schedule of the two-region box.
//
// Particles live in device banks instead of registers, one array per field
// (structure of arrays).  Each iteration is ONE kernel that streams the
// current bank in slot order -- every field load of a warp is one coalesced
// access -- and moves each particle one event: it flies, and if it stops at
// a collision site it collides.  Survivors are appended to the other bank
// (one atomic per group of converged lanes, so a group's stores land in
// consecutive slots), which keeps the bank dense: no dead slots, no queue.
// A particle that ended (leak, roulette, event cap) is replaced in the same
// pass by the next item of the generation from a ticket (a source history
// or a split child), so the bank stays full while there is work.  The block
// that finishes last (a counter, no waiting) swaps the banks and sets the
// completion flag.  The host launches iterations in batches (optionally one
// captured graph per batch) and reads the flag between batches; no kernel
// waits on another.
//
// Split children go to a device child bank and are followed as the next
// generation, exactly as in the history schedule.  Once every item of a
// generation has started and the live particles no longer fill the GPU, one
// tail kernel runs each live particle to its end.  All per-particle
// arithmetic is box.cuh's (the same draws, in the same order, and the same
// int64 contributions), so the mesh tally is bit-identical to the history
// schedule's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "box.cuh"
#include "internal.h"
#include "transport.h"

namespace {

using mcb::BoxDev;
using mcb::ChildRec;

struct Ctl {
  unsigned int n[2];           // particles in each bank
  unsigned int cur;            // the bank the next iteration reads
  unsigned int done;           // 1: generation finished; 2: tail kernel next
  unsigned int blocks_done;    // blocks of the running iteration that finished
  unsigned int pad;
  unsigned long long ticket;   // next item of the generation
  unsigned long long iters;
};

// One bank: an array per field.  T = float: 88 bytes per particle;
// T = double: 128.
template <typename T>
struct SoA {
  T *p[3], *u[3], *inv[3], *w;
  uint64_t *rng, *draws, *events, *gi, *tbase;
  uint32_t *prob, *flags;  // flags: group | region << 8 | primary << 16
};

template <typename T>
struct Bank {
  Ctl* ctl;
  mcd::Affine* tab;  // maps of 2^j LCG steps (stride seeding)
  SoA<T> f[2];
  uint32_t cap;
};

template <typename T>
struct Args {
  uint32_t tail_threshold;   // live particles at or below which the tail kernel takes over
  const BoxDev* probs;
  uint32_t nprob;
  const ChildRec* child_in;  // nullptr: the items are source histories
  uint64_t range_begin, total;
  ChildRec* child_out;
  unsigned long long* child_out_count;
  uint64_t child_cap;
  unsigned long long* tally;
  unsigned long long* counts;
  uint64_t* hist_state;
  uint64_t* hist_draws;
  mcd::Lcg lcg;
  uint64_t event_cap;
  Bank<T> b;
};

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

template <typename T>
size_t carve(void* base, uint32_t cap, Bank<T>* out) {
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += a256(bytes);
    return q;
  };
  Bank<T> b{};
  b.ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  b.tab = reinterpret_cast<mcd::Affine*>(take(64 * sizeof(mcd::Affine)));
  for (int k = 0; k < 2; ++k) {
    SoA<T>& f = b.f[k];
    for (int a = 0; a < 3; ++a) {
      f.p[a] = reinterpret_cast<T*>(take((size_t)cap * sizeof(T)));
      f.u[a] = reinterpret_cast<T*>(take((size_t)cap * sizeof(T)));
      f.inv[a] = reinterpret_cast<T*>(take((size_t)cap * sizeof(T)));
    }
    f.w = reinterpret_cast<T*>(take((size_t)cap * sizeof(T)));
    uint64_t** uu[] = {&f.rng, &f.draws, &f.events, &f.gi, &f.tbase};
    for (uint64_t** x : uu) *x = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
    f.prob = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
    f.flags = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
  }
  b.cap = cap;
  if (out) *out = b;
  return off;
}

// A particle as the kernels hold it.
template <typename T>
struct Live {
  mcb::Part<T> q;
  uint64_t rng, draws, events, gi, tbase;
  uint32_t prob, primary;
};

template <typename T>
__device__ __forceinline__ void load_live(const SoA<T>& f, uint32_t s, Live<T>& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v.q.p[a] = f.p[a][s];
    v.q.u[a] = f.u[a][s];
    v.q.inv[a] = f.inv[a][s];
  }
  v.q.w = f.w[s];
  v.rng = f.rng[s];
  v.draws = f.draws[s];
  v.events = f.events[s];
  v.gi = f.gi[s];
  v.tbase = f.tbase[s];
  v.prob = f.prob[s];
  const uint32_t fl = f.flags[s];
  v.q.g = fl & 0xffu;
  v.q.region = (fl >> 8) & 0xffu;
  v.primary = fl >> 16;
}

template <typename T>
__device__ __forceinline__ void store_live(const SoA<T>& f, uint32_t s, const Live<T>& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f.p[a][s] = v.q.p[a];
    f.u[a][s] = v.q.u[a];
    f.inv[a][s] = v.q.inv[a];
  }
  f.w[s] = v.q.w;
  f.rng[s] = v.rng;
  f.draws[s] = v.draws;
  f.events[s] = v.events;
  f.gi[s] = v.gi;
  f.tbase[s] = v.tbase;
  f.prob[s] = v.prob;
  f.flags[s] = v.q.g | (v.q.region << 8) | (v.primary << 16);
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

// The next item of the generation for each converged lane that asks (one
// atomic per group); a value >= total once the ticket has run out.
__device__ __forceinline__ unsigned long long take_item(unsigned long long* ticket) {
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned rank = __popc(mask & ((1u << lane) - 1u));
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(ticket, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + rank;
}

__device__ __forceinline__ uint32_t find_box(const BoxDev* p, uint32_t n, uint64_t gi) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (p[mid].hist_begin <= gi) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Starts item `item` of the generation in `v` (a source history: its seed
// and source sample; a child: its record from the child bank).
template <int M, typename T>
__device__ __forceinline__ void start_item(const Args<T>& a, const mcd::Affine* tab, uint64_t item, Live<T>& v) {
  mcs::Rng<M> r{0ull, 0ull};
  v.q = mcb::Part<T>{};
  if (a.child_in == nullptr) {
    const uint64_t gi = a.range_begin + item;
    const uint32_t pi = a.nprob == 1 ? 0u : find_box(a.probs, a.nprob, gi);
    const BoxDev& P = a.probs[pi];
    const uint64_t id = gi - P.hist_begin;
    const uint64_t nvox = (uint64_t)P.mesh * P.mesh * P.mesh;
    const uint64_t seed = P.seeding == MC_SEED_STRIDE
                              ? mcs::skip_tab(tab, P.seed, P.stride_q * (P.id_offset + id)) & a.lcg.mask
                              : mcd::hash_with(id, P.seed_hash) & a.lcg.mask;
    r = mcs::Rng<M>{seed, 0ull};
    mcb::box_source<M, T>(P, r, a.lcg, v.q);
    v.gi = gi;
    v.tbase = P.tally_offset + mcs::batch_of(id, P.n_hist, P.n_batches) * nvox;
    v.prob = pi;
    v.primary = 1u;
  } else {
    const ChildRec cr = a.child_in[item];
    r = mcs::Rng<M>{cr.rng, 0ull};
    mcb::load_child<T>(cr, v.q);
    v.gi = 0;
    v.tbase = cr.tbase;
    v.prob = cr.prob;
    v.primary = 0u;
  }
  v.rng = r.x;
  v.draws = r.draws;
  v.events = 0;
}

// The end of a particle: counters into the thread's `ec` (flushed by its
// warp at the end of the kernel, or here when the problem changes) and the
// per-history outputs of a source history.  outcome: kBoxLeak, kBoxKilled
// or -1 (event cap).
template <typename T>
__device__ void finish(const Args<T>& a, const BoxDev& P, const Live<T>& v, int outcome, mcb::BoxCounts& ec) {
  if ((int)v.prob != ec.prob) { ec.flush(a.counts); ec.prob = (int)v.prob; }
  const bool prim = v.primary != 0u;
  if (prim) ++ec.src;
  if (outcome == mcb::kBoxLeak) ++ec.leaks;
  else if (outcome == mcb::kBoxKilled) ++ec.kills;
  else ++ec.capped;
  ec.draws += v.draws;
  if (v.draws > ec.maxd) ec.maxd = v.draws;
  if (prim) {
    if (P.stride_q != 0 && v.draws > P.stride_q) {
      ++ec.exh;
      ec.exd += v.draws - P.stride_q;
    }
    if (a.hist_state) a.hist_state[v.gi] = v.rng & a.lcg.mask;
    if (a.hist_draws) a.hist_draws[v.gi] = v.draws;
  }
  if (ec.draws > (1ull << 31) || ec.flights > (1u << 30)) ec.flush(a.counts);
}

// Split children of the collision just made go to the next generation.
template <typename T>
__device__ __forceinline__ void bank_children(const Args<T>& a, int c, const mcb::Part<T>& q, uint64_t rng,
                                              uint32_t prob, uint64_t tbase, mcb::BoxCounts& ec) {
  const uint32_t ns = (uint32_t)(c - mcb::kSplitBase);
  ++ec.splits;
  ec.children += ns - 1;
  for (uint32_t k = 0; k + 1 < ns; ++k) {
    const unsigned long long idx = atomicAdd(a.child_out_count, 1ull);
    if (idx < a.child_cap) mcb::store_child<T>(a.child_out[idx], q, mcb::child_seed(k, rng, a.lcg.mask), prob, tbase);
  }
}

// Shared-memory copies of a single problem's record and (fp64) mesh planes,
// read on every flight and voxel crossing.
template <typename T>
struct SharedProblem {
  unsigned char prob[sizeof(BoxDev)];
  double planes[sizeof(T) == 8 ? mcb::kMaxPlanes : 1];
};

template <typename T>
__device__ __forceinline__ const BoxDev* stage_problem(const Args<T>& a, SharedProblem<T>& sp,
                                                       const double** planes) {
  *planes = nullptr;
  if (a.nprob != 1) return a.probs;
  const uint64_t* src = reinterpret_cast<const uint64_t*>(a.probs);
  uint64_t* dst = reinterpret_cast<uint64_t*>(sp.prob);
  for (uint32_t i = threadIdx.x; i < sizeof(BoxDev) / 8; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  const BoxDev* p = reinterpret_cast<const BoxDev*>(sp.prob);
  if constexpr (sizeof(T) == 8) {
    for (uint32_t j = threadIdx.x; j <= p->mesh; j += blockDim.x) sp.planes[j] = mcb::plane_of(*p, (int)j);
    __syncthreads();
    *planes = sp.planes;
  }
  return p;
}

// First pass of a generation: the first min(cap, total) items into bank 0,
// and the control block reset.
template <int M, typename T>
__global__ void __launch_bounds__(256) init_kernel(Args<T> a) {
  __shared__ mcd::Affine tab[64];
  if (threadIdx.x == 0) {
    mcd::Affine sq{a.lcg.g, a.lcg.c};
    for (int j = 0; j < 64; ++j) { tab[j] = sq; sq = mcd::compose(sq, sq); }
  }
  __syncthreads();
  const Bank<T>& b = a.b;
  const uint64_t n = a.total < b.cap ? a.total : b.cap;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < n; i += nt) {
    Live<T> v;
    start_item<M, T>(a, tab, i, v);
    store_live<T>(b.f[0], (uint32_t)i, v);
  }
  if (tid == 0) {
    Ctl* c = b.ctl;
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

// One iteration: every particle of the current bank flies once and, at a
// collision site, collides; survivors, and the items that replace ended
// particles, go to the other bank.  The last block to finish advances the
// control block.
template <int M, typename T>
__global__ void __launch_bounds__(256, 4) step_kernel(Args<T> a) {
  __shared__ __align__(16) SharedProblem<T> sp;
  const double* planes = nullptr;
  const BoxDev* probs = stage_problem<T>(a, sp, &planes);
  const Bank<T>& b = a.b;
  Ctl* c = b.ctl;
  const unsigned int cur = c->cur;
  const uint32_t n = c->n[cur];
  const SoA<T>& fin = b.f[cur];
  const SoA<T>& fout = b.f[cur ^ 1u];
  unsigned int* nout = &c->n[cur ^ 1u];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  mcb::BoxCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    Live<T> v;
    load_live<T>(fin, (uint32_t)t, v);
    const BoxDev& P = probs[v.prob];
    mcs::Rng<M> r{v.rng, v.draws};
    int outcome = -2;  // -2: alive after this iteration
    if (v.events == a.event_cap) {
      outcome = -1;
    } else {
      ++v.events;
      if ((int)v.prob != ec.prob) { ec.flush(a.counts); ec.prob = (int)v.prob; }
      ++ec.flights;
      const int o = mcb::box_flight<M, T>(P, r, a.lcg, v.q, a.tally + v.tbase, planes, false);
      if (o == mcb::kBoxLeak) {
        outcome = o;
      } else if (o == mcb::kBoxCollide) {
        ++ec.coll;
        const int cc = mcb::box_collide<M, T>(P, r, a.lcg, v.q);
        if (cc == mcb::kBoxKilled) outcome = cc;
        else if (cc >= mcb::kSplitBase + 2) bank_children<T>(a, cc, v.q, r.x, v.prob, v.tbase, ec);
      }
    }
    v.rng = r.x;
    v.draws = r.draws;
    bool keep = true;
    if (outcome != -2) {
      finish<T>(a, P, v, outcome, ec);
      const unsigned long long item = take_item(&c->ticket);
      if (item < a.total) start_item<M, T>(a, b.tab, item, v);
      else keep = false;
    }
    if (keep) store_live<T>(fout, take_slot(nout), v);
  }
  ec.flush_warp(a.counts);
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

// The tail of a generation: each particle of the current bank flies,
// crosses and collides to its end in one thread.
template <int M, typename T>
__global__ void __launch_bounds__(256, 3) tail_kernel(Args<T> a) {
  __shared__ __align__(16) SharedProblem<T> sp;
  const double* planes = nullptr;
  const BoxDev* probs = stage_problem<T>(a, sp, &planes);
  const Bank<T>& b = a.b;
  const unsigned int cur = b.ctl->cur;
  const uint32_t n = b.ctl->n[cur];
  const SoA<T>& fin = b.f[cur];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  mcb::BoxCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    Live<T> v;
    load_live<T>(fin, (uint32_t)t, v);
    const BoxDev& P = probs[v.prob];
    mcs::Rng<M> r{v.rng, v.draws};
    unsigned long long* const base = a.tally + v.tbase;
    if ((int)v.prob != ec.prob) { ec.flush(a.counts); ec.prob = (int)v.prob; }
    int outcome;
    for (;;) {
      if (v.events == a.event_cap) { outcome = -1; break; }
      ++v.events;
      ++ec.flights;
      const int o = mcb::box_flight<M, T>(P, r, a.lcg, v.q, base, planes, false);
      if (o == mcb::kBoxLeak) { outcome = o; break; }
      if (o != mcb::kBoxCollide) continue;  // crossed into the other region
      ++ec.coll;
      const int cc = mcb::box_collide<M, T>(P, r, a.lcg, v.q);
      if (cc == mcb::kBoxKilled) { outcome = cc; break; }
      if (cc >= mcb::kSplitBase + 2) bank_children<T>(a, cc, v.q, r.x, v.prob, v.tbase, ec);
    }
    v.rng = r.x;
    v.draws = r.draws;
    finish<T>(a, P, v, outcome, ec);
  }
  ec.flush_warp(a.counts);
}

constexpr int kIter = 32;

template <int M, typename T>
void enqueue_batch(const Args<T>& a, int grid, cudaStream_t s) {
  for (int k = 0; k < kIter; ++k) step_kernel<M, T><<<grid, 256, 0, s>>>(a);
}

// Runs one generation (sources or children) to completion.
template <int M, typename T>
int run_generation(const Args<T>& a, int grid, uint64_t max_batches, const mci::BoxLaunch& L, cudaStream_t s) {
  init_kernel<M, T><<<grid, 256, 0, s>>>(a);
  MC_TRY_CUDA(cudaGetLastError());
  cudaGraphExec_t exec = nullptr;
  if (L.capture_stream) {
    cudaGraph_t g = nullptr;
    MC_TRY_CUDA(cudaStreamBeginCapture(L.capture_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_batch<M, T>(a, grid, L.capture_stream);
    cudaError_t e = cudaStreamEndCapture(L.capture_stream, &g);
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaStreamEndCapture(box event batch)");
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return mci::cuda_status(e, "cudaGraphInstantiate(box event batch)");
  }
  int st = MC_OK;
  for (uint64_t batch = 0;; ++batch) {
    // the completion flag as the init kernel or the last iteration left it
    cudaError_t e = cudaMemcpyAsync(L.h_done, &a.b.ctl->done, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = mci::cuda_status(e, "box event completion check");
      break;
    }
    if (*L.h_done == 2u) {  // the rest of the generation in one kernel
      tail_kernel<M, T><<<grid, 256, 0, s>>>(a);
      st = mci::cuda_status(cudaGetLastError(), "box tail_kernel launch");
      break;
    }
    if (*L.h_done) break;
    if (batch == max_batches) {
      mci::set_error("box event schedule: no completion after %llu iterations",
                     (unsigned long long)(batch * kIter));
      st = MC_ERR_TIMEOUT;
      break;
    }
    if (exec) {
      e = cudaGraphLaunch(exec, s);
    } else {
      enqueue_batch<M, T>(a, grid, s);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      st = mci::cuda_status(e, "box event batch");
      break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  return st;
}

template <int M, typename T>
int run_box_event(const mci::BoxLaunch& L, cudaStream_t s) {
  Args<T> a{};
  a.probs = static_cast<const BoxDev*>(L.d_probs);
  a.nprob = L.n_problems;
  a.child_cap = L.child_cap;
  a.tally = reinterpret_cast<unsigned long long*>(L.tally->d_bins);
  a.counts = reinterpret_cast<unsigned long long*>(L.tally->d_counts);
  a.hist_state = L.tally->d_hist_state;
  a.hist_draws = L.tally->d_hist_draws;
  a.lcg = mcd::Lcg{L.lcg.g, L.lcg.c, mcd::mask_of(L.lcg.m), L.lcg.m};
  a.event_cap = L.event_cap;
  carve<T>(L.d_bank, L.bank_cap, &a.b);
  // One wave of resident blocks: every block of an iteration runs at once.
  int per_sm = 0;
  MC_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<M, T>, 256, 0));
  const int grid = std::max(1, L.num_sms * std::max(per_sm, 1));
  // Box particles live a few dozen flights: once the ticket is spent, a
  // half-empty bank is finished faster by the tail kernel than by
  // iterations of ever fewer particles.
  a.tail_threshold = std::max<uint32_t>((uint32_t)L.num_sms * 1024u, L.bank_cap / 2);
  // Each iteration moves every live particle one event and the bank refills
  // from the ticket; the bound below is a safety net only.
  uint64_t max_batches = (std::min<uint64_t>(L.event_cap, 1ull << 36) * 4 + 64) / kIter +
                         (L.total / std::max<uint32_t>(L.bank_cap, 1u) + 2) * 4;
  if (L.event_iterations != ~0ull)  // a caller's bound (mc_limits), in whole batches
    max_batches = L.event_iterations / kIter + (L.event_iterations % kIter != 0);
  ChildRec* bank[2] = {static_cast<ChildRec*>(L.d_child[0]), static_cast<ChildRec*>(L.d_child[1])};
  unsigned long long* cnt[2] = {L.d_child_count, L.d_child_count + 1};
  for (uint64_t start = 0; start < L.total; start += L.primary_chunk) {
    const uint64_t n = std::min<uint64_t>(L.primary_chunk, L.total - start);
    MC_TRY_CUDA(cudaMemsetAsync(cnt[0], 0, sizeof(unsigned long long), s));
    a.child_in = nullptr;
    a.range_begin = L.range_begin + start;
    a.total = n;
    a.child_out = bank[0];
    a.child_out_count = cnt[0];
    int st = run_generation<M, T>(a, grid, max_batches, L, s);
    if (st != MC_OK) return st;
    int cur = 0;
    for (int gen = 1;; ++gen) {
      MC_TRY_CUDA(cudaMemcpyAsync(L.h_count, cnt[cur], sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      MC_TRY_CUDA(cudaStreamSynchronize(s));
      const unsigned long long made = *L.h_count;
      if (made > L.child_cap) {
        mci::set_error("box event schedule: %llu children exceed the bank of %llu", made,
                       (unsigned long long)L.child_cap);
        return MC_ERR_CAPACITY;
      }
      if (made == 0) break;
      if ((uint32_t)gen > L.max_generations) {
        mci::set_error("box event schedule: more than %u generations", L.max_generations);
        return MC_ERR_TIMEOUT;
      }
      const int nxt = cur ^ 1;
      MC_TRY_CUDA(cudaMemsetAsync(cnt[nxt], 0, sizeof(unsigned long long), s));
      a.child_in = bank[cur];
      a.range_begin = 0;
      a.total = made;
      a.child_out = bank[nxt];
      a.child_out_count = cnt[nxt];
      st = run_generation<M, T>(a, grid, max_batches, L, s);
      if (st != MC_OK) return st;
      cur = nxt;
    }
  }
  return MC_OK;
}

}  // namespace

namespace mci {

size_t box_bank_bytes(uint32_t cap) {
  return std::max(carve<double>(nullptr, cap, nullptr), carve<float>(nullptr, cap, nullptr));
}

int box_event_run(const BoxLaunch& L, cudaStream_t s) {
  if (L.lcg.m == 63) return L.f32 ? run_box_event<63, float>(L, s) : run_box_event<63, double>(L, s);
  return L.f32 ? run_box_event<0, float>(L, s) : run_box_event<0, double>(L, s);
}

}  // namespace mci

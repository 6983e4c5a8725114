// box_event.cu -- event-based schedule of the two-region box.
//
// Same structure as the slab event schedule: particles in a device bank,
// one kernel per event type over queues of bank slots (plan, refill,
// flight, collide, advance), iterations launched in batches by the host
// (optionally as a captured graph).  Split children go to a device child
// bank and are followed as the next generation, exactly as in the history
// schedule.  All per-particle arithmetic is box.cuh's, so the int64 mesh
// tally is bit-identical to the history schedule's.
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
  unsigned int nfq[2], ncq, nfree, cur, refill_n, refill_free_base, done;
  unsigned long long refill_ticket_base, ticket, iters;
};

struct Bank {
  Ctl* ctl;
  mcd::Affine* tab;
  double *px, *py, *pz, *ux, *uy, *uz, *w;
  uint64_t *rng, *draws, *events, *gi, *tbase;
  uint32_t *prob, *grp, *region, *primary, *coll;
  uint32_t *fq0, *fq1, *cq, *freeq;
  uint32_t cap;
};

struct Args {
  uint32_t tail_threshold;  // live particles at or below which the tail kernel takes over
  const BoxDev* probs;
  uint32_t nprob;
  const ChildRec* child_in;  // nullptr: source histories
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
  Bank b;
};

size_t a256(size_t v) { return (v + 255) & ~size_t(255); }

size_t carve(void* base, uint32_t cap, Bank* out) {
  char* p = static_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += a256(bytes);
    return q;
  };
  Bank b{};
  b.ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  b.tab = reinterpret_cast<mcd::Affine*>(take(64 * sizeof(mcd::Affine)));
  double** dd[] = {&b.px, &b.py, &b.pz, &b.ux, &b.uy, &b.uz, &b.w};
  for (double** d : dd) *d = reinterpret_cast<double*>(take((size_t)cap * 8));
  uint64_t** uu[] = {&b.rng, &b.draws, &b.events, &b.gi, &b.tbase};
  for (uint64_t** u : uu) *u = reinterpret_cast<uint64_t*>(take((size_t)cap * 8));
  uint32_t** ii[] = {&b.prob, &b.grp, &b.region, &b.primary, &b.coll, &b.fq0, &b.fq1, &b.cq, &b.freeq};
  for (uint32_t** i : ii) *i = reinterpret_cast<uint32_t*>(take((size_t)cap * 4));
  b.cap = cap;
  if (out) *out = b;
  return off;
}

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

template <typename T>
__device__ __forceinline__ void load_part(const Bank& b, uint32_t s, mcb::Part<T>& q) {
  q.p[0] = (T)b.px[s]; q.p[1] = (T)b.py[s]; q.p[2] = (T)b.pz[s];
  q.u[0] = (T)b.ux[s]; q.u[1] = (T)b.uy[s]; q.u[2] = (T)b.uz[s];
  q.w = (T)b.w[s];
  q.g = b.grp[s];
  q.region = b.region[s];
  mcb::set_inv(q);
}

template <typename T>
__device__ __forceinline__ void store_part(const Bank& b, uint32_t s, const mcb::Part<T>& q) {
  b.px[s] = (double)q.p[0]; b.py[s] = (double)q.p[1]; b.pz[s] = (double)q.p[2];
  b.ux[s] = (double)q.u[0]; b.uy[s] = (double)q.u[1]; b.uz[s] = (double)q.u[2];
  b.w[s] = (double)q.w;
  b.grp[s] = q.g;
  b.region[s] = q.region;
}

__global__ void init_kernel(Args a) {
  const Bank& b = a.b;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = tid; i < b.cap; i += nt) b.freeq[i] = (uint32_t)(b.cap - 1 - i);
  if (tid == 0) {
    Ctl* c = b.ctl;
    c->nfq[0] = c->nfq[1] = 0;
    c->ncq = 0;
    c->nfree = b.cap;
    c->cur = 0;
    c->refill_n = c->refill_free_base = 0;
    c->done = a.total == 0 ? 1u : 0u;
    c->refill_ticket_base = c->ticket = c->iters = 0;
    mcd::Affine sq{a.lcg.g, a.lcg.c};
    for (int j = 0; j < 64; ++j) { b.tab[j] = sq; sq = mcd::compose(sq, sq); }
  }
}

__global__ void plan_kernel(Args a) {
  Ctl* c = a.b.ctl;
  const uint64_t F = c->nfree, R = a.total - c->ticket;
  const uint64_t n = F < R ? F : R;
  c->refill_n = (unsigned int)n;
  c->refill_free_base = (unsigned int)(F - n);
  c->refill_ticket_base = c->ticket;
  c->nfree = (unsigned int)(F - n);
  c->ticket += n;
}

__device__ __forceinline__ uint32_t find_box(const BoxDev* p, uint32_t n, uint64_t gi) {
  uint32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (p[mid].hist_begin <= gi) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int M, typename T>
__global__ void __launch_bounds__(256) refill_kernel(Args a) {
  const Bank& b = a.b;
  const Ctl* c = b.ctl;
  const uint32_t n = c->refill_n, fb = c->refill_free_base;
  const uint64_t tb = c->refill_ticket_base;
  uint32_t* fq = c->cur ? b.fq1 : b.fq0;
  unsigned int* nfq = &b.ctl->nfq[c->cur];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t s = b.freeq[fb + t];
    const uint64_t item = tb + t;
    mcb::Part<T> q{};
    mcs::Rng<M> r{0ull, 0ull};
    uint32_t pi;
    if (a.child_in == nullptr) {
      const uint64_t gi = a.range_begin + item;
      pi = a.nprob == 1 ? 0u : find_box(a.probs, a.nprob, gi);
      const BoxDev& P = a.probs[pi];
      const uint64_t id = gi - P.hist_begin;
      const uint64_t nvox = (uint64_t)P.mesh * P.mesh * P.mesh;
      const uint64_t seed = P.seeding == MC_SEED_STRIDE
                                ? mcs::skip_tab(b.tab, P.seed, P.stride_q * (P.id_offset + id)) & a.lcg.mask
                                : mcd::hash_with(id, P.seed_hash) & a.lcg.mask;
      r = mcs::Rng<M>{seed, 0ull};
      mcb::box_source<M, T>(P, r, a.lcg, q);
      b.gi[s] = gi;
      b.tbase[s] = P.tally_offset + mcs::batch_of(id, P.n_hist, P.n_batches) * nvox;
      b.primary[s] = 1u;
    } else {
      const ChildRec cr = a.child_in[item];
      pi = cr.prob;
      r = mcs::Rng<M>{cr.rng, 0ull};
      mcb::load_child<T>(cr, q);
      b.gi[s] = 0;
      b.tbase[s] = cr.tbase;
      b.primary[s] = 0u;
    }
    b.prob[s] = pi;
    b.rng[s] = r.x;
    b.draws[s] = r.draws;
    b.events[s] = 0;
    b.coll[s] = 0;
    store_part<T>(b, s, q);
    warp_append(nfq, fq, s);
  }
}

// outcome: mcb::kBoxLeak, kBoxKilled, or -1 (event cap).  The particle's
// counts go to the thread's counters `ec` (flushed by its warp at the end of
// the kernel, or here when the problem changes).
__device__ void finish(const Args& a, uint32_t s, int outcome, uint64_t rng_x, uint64_t draws, mcb::BoxCounts& ec) {
  const Bank& b = a.b;
  const uint32_t pi = b.prob[s];
  const BoxDev& P = a.probs[pi];
  if ((int)pi != ec.prob) { ec.flush(a.counts); ec.prob = (int)pi; }
  const bool prim = b.primary[s] != 0u;
  if (prim) ++ec.src;
  ec.flights += (uint32_t)b.events[s];
  ec.coll += b.coll[s];
  if (outcome == mcb::kBoxLeak) ++ec.leaks;
  else if (outcome == mcb::kBoxKilled) ++ec.kills;
  else ++ec.capped;
  ec.draws += draws;
  if (draws > ec.maxd) ec.maxd = draws;
  if (prim) {
    if (P.stride_q != 0 && draws > P.stride_q) {
      ++ec.exh;
      ec.exd += draws - P.stride_q;
    }
    const uint64_t gi = b.gi[s];
    if (a.hist_state) a.hist_state[gi] = rng_x & a.lcg.mask;
    if (a.hist_draws) a.hist_draws[gi] = draws;
  }
  if (ec.draws > (1ull << 31) || ec.flights > (1u << 30)) ec.flush(a.counts);
  const unsigned int k = atomicAdd(&b.ctl->nfree, 1u);
  b.freeq[k] = s;
}

template <int M, typename T>
__global__ void __launch_bounds__(256) flight_kernel(Args a) {
  const Bank& b = a.b;
  const unsigned int cur = b.ctl->cur;
  const uint32_t n = b.ctl->nfq[cur];
  const uint32_t* fq = cur ? b.fq1 : b.fq0;
  uint32_t* fnext = cur ? b.fq0 : b.fq1;
  unsigned int* nnext = &b.ctl->nfq[cur ^ 1u];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  mcb::BoxCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t s = fq[t];
    const BoxDev& P = a.probs[b.prob[s]];
    mcs::Rng<M> r{b.rng[s], b.draws[s]};
    const uint64_t ev = b.events[s];
    if (ev == a.event_cap) {
      finish(a, s, -1, r.x, r.draws, ec);
      continue;
    }
    b.events[s] = ev + 1;
    mcb::Part<T> q;
    load_part<T>(b, s, q);
    const int o = mcb::box_flight<M, T>(P, r, a.lcg, q, a.tally + b.tbase[s], nullptr, false);
    if (o == mcb::kBoxLeak) {
      finish(a, s, o, r.x, r.draws, ec);
      continue;
    }
    b.rng[s] = r.x;
    b.draws[s] = r.draws;
    b.px[s] = (double)q.p[0]; b.py[s] = (double)q.p[1]; b.pz[s] = (double)q.p[2];
    b.region[s] = q.region;
    if (o == mcb::kBoxCollide) warp_append(&b.ctl->ncq, b.cq, s);
    else warp_append(nnext, fnext, s);
  }
  ec.flush_warp(a.counts);
}

template <int M, typename T>
__global__ void __launch_bounds__(256) collide_kernel(Args a) {
  const Bank& b = a.b;
  const unsigned int nxt = b.ctl->cur ^ 1u;
  const uint32_t n = b.ctl->ncq;
  uint32_t* fq = nxt ? b.fq1 : b.fq0;
  unsigned int* nfq = &b.ctl->nfq[nxt];
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  mcb::BoxCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t s = b.cq[t];
    const uint32_t pi = b.prob[s];
    const BoxDev& P = a.probs[pi];
    mcs::Rng<M> r{b.rng[s], b.draws[s]};
    mcb::Part<T> q;
    load_part<T>(b, s, q);
    b.coll[s] += 1u;
    const int o = mcb::box_collide<M, T>(P, r, a.lcg, q);
    if (o == mcb::kBoxKilled) {
      finish(a, s, o, r.x, r.draws, ec);
      continue;
    }
    if (o >= mcb::kSplitBase + 2) {
      const uint32_t ns = (uint32_t)(o - mcb::kSplitBase);
      if ((int)pi != ec.prob) { ec.flush(a.counts); ec.prob = (int)pi; }
      ++ec.splits;
      ec.children += ns - 1;
      for (uint32_t k = 0; k + 1 < ns; ++k) {
        const unsigned long long idx = atomicAdd(a.child_out_count, 1ull);
        if (idx < a.child_cap)
          mcb::store_child<T>(a.child_out[idx], q, mcb::child_seed(k, r.x, a.lcg.mask), pi, b.tbase[s]);
      }
    }
    b.rng[s] = r.x;
    b.draws[s] = r.draws;
    store_part<T>(b, s, q);
    warp_append(nfq, fq, s);
  }
  ec.flush_warp(a.counts);
}

__global__ void advance_kernel(Args a) {
  Ctl* c = a.b.ctl;
  const unsigned int cur = c->cur;
  c->nfq[cur] = 0;
  c->ncq = 0;
  c->cur = cur ^ 1u;
  const unsigned int live = c->nfq[cur ^ 1u];
  // 1: finished; 2: every particle of the generation started and few enough
  // live for the tail kernel
  c->done = c->ticket < a.total ? 0u : (live == 0 ? 1u : (live <= a.tail_threshold ? 2u : 0u));
  c->iters += 1;
}

// The tail of a generation: each live particle of the current flight queue
// flies, crosses and collides to its end in one thread (split children go
// to the child bank as in collide_kernel).
template <int M, typename T>
__global__ void __launch_bounds__(256) tail_kernel(Args a) {
  const Bank& b = a.b;
  const unsigned int cur = b.ctl->cur;
  const uint32_t n = b.ctl->nfq[cur];
  const uint32_t* fq = cur ? b.fq1 : b.fq0;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  mcb::BoxCounts ec;
  ec.prob = -1;
  ec.clear();
  for (uint64_t t = tid; t < n; t += nt) {
    const uint32_t s = fq[t];
    const uint32_t pi = b.prob[s];
    const BoxDev& P = a.probs[pi];
    mcs::Rng<M> r{b.rng[s], b.draws[s]};
    mcb::Part<T> q;
    load_part<T>(b, s, q);
    unsigned long long* const base = a.tally + b.tbase[s];
    uint64_t ev = b.events[s];
    uint32_t co = b.coll[s];
    int outcome;
    for (;;) {
      if (ev == a.event_cap) { outcome = -1; break; }
      ++ev;
      const int o = mcb::box_flight<M, T>(P, r, a.lcg, q, base, nullptr, false);
      if (o == mcb::kBoxLeak) { outcome = o; break; }
      if (o != mcb::kBoxCollide) continue;  // crossed into the other region
      ++co;
      const int c = mcb::box_collide<M, T>(P, r, a.lcg, q);
      if (c == mcb::kBoxKilled) { outcome = c; break; }
      if (c >= mcb::kSplitBase + 2) {
        const uint32_t ns = (uint32_t)(c - mcb::kSplitBase);
        if ((int)pi != ec.prob) { ec.flush(a.counts); ec.prob = (int)pi; }
        ++ec.splits;
        ec.children += ns - 1;
        for (uint32_t k = 0; k + 1 < ns; ++k) {
          const unsigned long long idx = atomicAdd(a.child_out_count, 1ull);
          if (idx < a.child_cap)
            mcb::store_child<T>(a.child_out[idx], q, mcb::child_seed(k, r.x, a.lcg.mask), pi, b.tbase[s]);
        }
      }
    }
    b.events[s] = ev;
    b.coll[s] = co;
    finish(a, s, outcome, r.x, r.draws, ec);
  }
  ec.flush_warp(a.counts);
}

constexpr int kIter = 32;

template <int M, typename T>
void enqueue_batch(const Args& a, int grid, cudaStream_t s) {
  for (int k = 0; k < kIter; ++k) {
    plan_kernel<<<1, 1, 0, s>>>(a);
    refill_kernel<M, T><<<grid, 256, 0, s>>>(a);
    flight_kernel<M, T><<<grid, 256, 0, s>>>(a);
    collide_kernel<M, T><<<grid, 256, 0, s>>>(a);
    advance_kernel<<<1, 1, 0, s>>>(a);
  }
}

// Runs one generation (sources or children) to completion.
template <int M, typename T>
int run_generation(const Args& a, int grid, const mci::BoxLaunch& L, cudaStream_t s) {
  init_kernel<<<grid, 256, 0, s>>>(a);
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
  uint64_t max_batches = (std::min<uint64_t>(L.event_cap, 1ull << 36) * 4 + 64) / kIter +
                         (a.total / a.b.cap + 2) * 4;
  if (L.event_iterations != ~0ull)  // a caller's bound (mc_limits), in whole batches
    max_batches = L.event_iterations / kIter + (L.event_iterations % kIter != 0);
  int st = MC_OK;
  for (uint64_t batch = 0;; ++batch) {
    if (batch == max_batches) {
      mci::set_error("box event schedule: no completion after %llu iterations",
                     (unsigned long long)(batch * kIter));
      st = MC_ERR_TIMEOUT;
      break;
    }
    cudaError_t e;
    if (exec) {
      e = cudaGraphLaunch(exec, s);
    } else {
      enqueue_batch<M, T>(a, grid, s);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(L.h_done, &a.b.ctl->done, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = mci::cuda_status(e, "box event batch");
      break;
    }
    if (*L.h_done == 2u) {  // the rest of the generation in one kernel
      tail_kernel<M, T><<<grid, 256, 0, s>>>(a);
      st = mci::cuda_status(cudaGetLastError(), "box tail_kernel launch");
      break;
    }
    if (*L.h_done) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  return st;
}

template <int M, typename T>
int run_box_event(const mci::BoxLaunch& L, cudaStream_t s) {
  Args a{};
  a.probs = static_cast<const BoxDev*>(L.d_probs);
  a.nprob = L.n_problems;
  a.child_cap = L.child_cap;
  a.tally = reinterpret_cast<unsigned long long*>(L.tally->d_bins);
  a.counts = reinterpret_cast<unsigned long long*>(L.tally->d_counts);
  a.hist_state = L.tally->d_hist_state;
  a.hist_draws = L.tally->d_hist_draws;
  a.lcg = mcd::Lcg{L.lcg.g, L.lcg.c, mcd::mask_of(L.lcg.m), L.lcg.m};
  a.event_cap = L.event_cap;
  carve(L.d_bank, L.bank_cap, &a.b);
  const int grid = std::max(1, L.num_sms * 4);
  a.tail_threshold = (uint32_t)L.num_sms * 1024u;
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
    int st = run_generation<M, T>(a, grid, L, s);
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
      st = run_generation<M, T>(a, grid, L, s);
      if (st != MC_OK) return st;
      cur = nxt;
    }
  }
  return MC_OK;
}

}  // namespace

namespace mci {

size_t box_bank_bytes(uint32_t cap) { return carve(nullptr, cap, nullptr); }

int box_event_run(const BoxLaunch& L, cudaStream_t s) {
  if (L.lcg.m == 63) return L.f32 ? run_box_event<63, float>(L, s) : run_box_event<63, double>(L, s);
  return L.f32 ? run_box_event<0, float>(L, s) : run_box_event<0, double>(L, s);
}

}  // namespace mci

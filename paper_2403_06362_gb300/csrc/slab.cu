// slab.cu -- persistent history-based slab transport and the host side of
// mc_transport_run.
//
// One lane carries one history at a time: its LCG state, position and
// direction stay in registers.  Each loop iteration every live lane flies
// one flight (and collides once); a lane whose history ended refills from
// its warp's chunk of history indices, and the warp leader takes a new chunk
// from a global ticket when the chunk runs dry.  So a warp keeps all 32
// lanes busy until the ticket is exhausted, however uneven the histories.
//
// Tallies are int64 fixed point (2^32), staged in shared memory when the
// whole tally fits and flushed with one global atomic per nonzero slot per
// block; otherwise contributions go straight to global atomics.  Counters
// are accumulated per lane and flushed when a lane changes problem.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"
#include "slab.cuh"
#include "transport.h"

namespace {

using mcs::SlabDev;

// Bin edge and width tables of every problem, after the records (`tables`
// may be null: no tables).
__global__ void slab_tables_kernel(const SlabDev* __restrict__ p, uint32_t n, double* __restrict__ tables) {
  for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
    const SlabDev& q = p[i];
    double* e = tables + q.tab_off;
    double* w = e + q.n_bins + 1;
    for (uint32_t j = threadIdx.x; j <= q.n_bins; j += blockDim.x) e[j] = mcs::slab_edge(q, (int)j);
    for (uint32_t j = threadIdx.x; j < q.n_bins; j += blockDim.x)
      w[j] = __dsub_rn(mcs::slab_edge(q, (int)j + 1), mcs::slab_edge(q, (int)j));
  }
}

// Expected flights per history of a slab problem with a uniform isotropic
// source, a ranking key only: the first-flight escape probability of such a
// source in a slab of optical thickness tau is (1 - 2 E3(tau)) / (2 tau)
// (E3 approximated by exp(-tau) / (tau + 2)), every later flight is taken to
// escape as often, and a collision continues with probability c:
// 1 / (1 - c (1 - P_esc)).
__device__ __forceinline__ float expected_flights(const SlabDev& q) {
  const float tau = fmaxf((float)(q.L * q.sigma_t), 1e-6f);
  const float e3 = __expf(-tau) / (tau + 2.0f);
  const float p_esc = fminf(1.0f, (1.0f - 2.0f * e3) / (2.0f * tau));
  return 1.0f / fmaxf(1e-6f, 1.0f - (float)q.c * (1.0f - p_esc));
}

__global__ void slab_prep_kernel(SlabDev* __restrict__ p, uint32_t n, uint32_t* __restrict__ order,
                                 uint64_t* __restrict__ order_begin) {
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    SlabDev& q = p[i];
    q.h = q.L / (double)q.n_bins;
    q.inv_h = (double)q.n_bins / q.L;
    mcx::fixed_of(q.inv_h, q.ih_q, q.ih_s);
    q.inv_st = 1.0 / q.sigma_t;
    q.p_abs = 1.0 - q.c;
    q.p_abs_n = (uint64_t)ceil(q.p_abs * 0x1p53);
    q.L_f = (float)q.L;
    q.h_f = q.L_f / (float)q.n_bins;
    q.inv_h_f = (float)q.n_bins / q.L_f;
    q.inv_st_f = 1.0f / (float)q.sigma_t;
    q.guard_f = q.L_f * 0x1p-18f;
    const uint64_t parent = q.seeding == MC_SEED_HASH_HIER ? mcd::hash64(q.key, q.seed) : q.seed;
    q.seed_hash = mcd::seed_hash_of(parent);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t acc = 0;
    for (uint32_t i = 0; i < n; ++i) {
      p[i].hist_begin = acc;
      acc += p[i].n_hist;
    }
  }
  if (!order) return;
  // rank by expected flights, descending; ties by index (a stable order)
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float fi = expected_flights(p[i]);
    uint32_t r = 0;
    for (uint32_t j = 0; j < n; ++j) {
      const float fj = expected_flights(p[j]);
      r += (fj > fi || (fj == fi && j < i)) ? 1u : 0u;
    }
    order[r] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t acc = 0;
    for (uint32_t k = 0; k < n; ++k) {
      order_begin[k] = acc;
      acc += p[order[k]].n_hist;
    }
    order_begin[n] = acc;
  }
}

struct RunArgs {
  const SlabDev* probs;
  uint32_t nprob;
  uint32_t chunk;
  uint64_t range_begin, total;
  unsigned long long* ticket;
  unsigned long long* tally;
  unsigned long long* counts;
  uint64_t* hist_state;
  uint64_t* hist_draws;
  mcd::Lcg lcg;
  uint64_t event_cap;
  uint32_t smem_slots;
  uint32_t smem_edges;  // single-problem launches: n_bins + 1 edges in shared memory (0: none)
  const double* tables; // else per-problem edge and width tables in global memory (nullable)
  uint32_t donate_max;  // a warp with 1..donate_max live lanes after the ticket ran out donates them
  uint32_t pool_cap;    // particles the block's shared pool holds (0: no compaction)
  uint32_t lock_attempts;  // attempts at the pool lock before a warp gives up
  uint32_t coop_slots;     // event records of the cooperative tail the pool's memory holds
  mcs::Order order;        // processing order of several problems (empty: id order)
};

// In-block compaction of the long-chain tail.  Once the ticket runs out,
// lanes whose histories end are no longer refilled and warps thin out (the
// fp64 slab ran at 4 live lanes of 32).  A warp left with few live lanes
// hands them to a shared-memory pool of its block and leaves the loop; warps
// with dead lanes take them from the pool.  A particle carries its whole
// state (stream, position, direction, history index, flight count), so the
// move changes no draw and no result.  The pool is guarded by a lock taken
// by one lane per warp, with bounded attempts; a warp that cannot take it
// skips the hand-over (or, leaving, counts the stranded particles in
// MC_C_DROPPED, the error the host reports).
constexpr int kPoolWords = 10;
struct PoolCtl {
  int lock, n, active, pad;
};

__device__ __forceinline__ bool pool_lock(int* lk, uint32_t attempts) {
  for (uint32_t i = 0; i < attempts; ++i)
    if (atomicCAS(lk, 0, 1) == 0) {
      __threadfence_block();
      return true;
    }
  return false;
}
__device__ __forceinline__ void pool_unlock(int* lk) {
  __threadfence_block();
  atomicExch(lk, 0);
}

template <int M>
__device__ __forceinline__ void pool_put(unsigned long long* e, const mcs::Rng<M>& r,
                                         const mcs::SlabParticle& q, uint64_t gi, uint64_t events,
                                         uint32_t pi) {
  e[0] = r.x;
  e[1] = r.draws;
  e[2] = (unsigned long long)__double_as_longlong(q.x);
  e[3] = (unsigned long long)__double_as_longlong(q.mu);
  e[4] = (unsigned long long)__double_as_longlong(q.w_mu);
  e[5] = ((unsigned long long)__float_as_uint(q.muf) << 32) | __float_as_uint(q.xf);
  e[6] = ((unsigned long long)pi << 32) | __float_as_uint(q.wf);
  e[7] = gi;
  e[8] = events;
  e[9] = __float_as_uint(q.xlo);
}

template <int M>
__device__ __forceinline__ uint32_t pool_get(const unsigned long long* e, mcs::Rng<M>& r, mcs::SlabParticle& q,
                                             uint64_t& gi, uint64_t& events) {
  r.x = e[0];
  r.draws = e[1];
  q.x = __longlong_as_double((long long)e[2]);
  q.mu = __longlong_as_double((long long)e[3]);
  q.w_mu = __longlong_as_double((long long)e[4]);
  q.xf = __uint_as_float((uint32_t)e[5]);
  q.muf = __uint_as_float((uint32_t)(e[5] >> 32));
  q.wf = __uint_as_float((uint32_t)e[6]);
  gi = e[7];
  events = e[8];
  q.xlo = __uint_as_float((uint32_t)e[9]);
  return (uint32_t)(e[6] >> 32);
}

// What the end of a history and the cooperative tail need of the launch.
struct TailArgs {
  uint64_t* hist_state;
  uint64_t* hist_draws;
  unsigned long long* counts;
  mcd::Lcg lcg;
  uint64_t event_cap;
};

// The cooperative tail's view of the launch.
struct CoopArgs {
  TailArgs t;
  const SlabDev* probs;
};

// End of a history: its draws into the lane's counters, its final state and
// draw count where the caller asked for them.
template <int M>
__device__ __forceinline__ void end_history(const TailArgs& t, const mcs::Rng<M>& r, const SlabDev* P, uint64_t gi,
                                            mcs::LaneCounts& lc) {
  lc.draws += r.draws;
  if (r.draws > lc.maxd) lc.maxd = r.draws;
  if (P->stride_q != 0 && r.draws > P->stride_q) { ++lc.exh; lc.exd += r.draws - P->stride_q; }
  if (t.hist_state) t.hist_state[gi] = r.x & t.lcg.mask;
  if (t.hist_draws) t.hist_draws[gi] = r.draws;
  if (lc.draws > (1ull << 31)) lc.flush(t.counts);
}

// Cooperative tail.  When the ticket has run out, the block's pool is empty
// and its last warp holds at most kCoopMax live histories, the rest of the
// launch is the latency of those few chains: one lane runs each, and a
// flight's dependent instructions (the logarithm of its uniform, its product
// with the direction, the absorption test, the next direction and its
// reciprocal) leave the other lanes idle.  But a history's draws have fixed
// roles -- each event takes one draw for the distance, one for the
// absorption test and one for the new direction, until the history ends --
// so everything that depends on the draws alone can be computed ahead.  The
// warp splits into one group of 32 / kp lanes per live history (kp: the live
// count rounded up to a power of two) and advances every history by rounds
// of E events:
//   1. the group's lanes compute, for each event e of the round, the
//      distance d_e, the product p_e = d_e mu_e, the absorption test and the
//      direction mu_{e+1} with its tally weight, jumping the stream to draw
//      3e with the maps of 2^j steps;
//   2. one lane runs the chain of positions alone, x_{e+1} = x_e + p_e and
//      the face tests, until the round ends or the history does (an event
//      cap, a leak, an absorption);
//   3. the group's lanes make the tally contributions of the round's events.
// Every value comes from the same function, with the same operands, as in
// the one-lane path, so the draws, tallies and counters are the same bits.
// The histories' state and the rounds' event records sit in the (then
// empty) pool's shared memory, the launch's arguments in a small shared
// record, and each phase is a function of its own that takes them from
// there: the main loop has ended, and almost nothing stays in registers
// across the calls.
constexpr int kCoopMax = 4;            // live histories at most
constexpr int kCoopHistWords = 16;     // 8-byte words per history record
constexpr int kCoopWords = 6;          // 8-byte words per event record
constexpr uint32_t kCoopEvents = 128;  // events per history and round at most
constexpr uint32_t kCoopMinEvents = 8;
// shared memory the tail's records get at least (words): room for rounds of
// kCoopEvents events with one history
constexpr size_t kCoopAreaWords = (size_t)kCoopMax * kCoopHistWords + (size_t)kCoopWords * (kCoopEvents + 1u);

__device__ __forceinline__ int coop_groups(int nlive) { return nlive <= 1 ? 1 : nlive <= 2 ? 2 : nlive <= 4 ? 4 : 8; }

__device__ __forceinline__ uint32_t coop_events(uint32_t slots, int kp) {
  const uint32_t per = slots / (uint32_t)kp;  // records per history: E events and the direction after them
  return per > 1u ? min(kCoopEvents, per - 1u) : 0u;
}

// Event records the pool's memory holds beside the history records.
__host__ __device__ __forceinline__ uint32_t coop_slots_of(uint32_t pool_words) {
  const uint32_t h = (uint32_t)(kCoopMax * kCoopHistWords);
  return pool_words > h ? (pool_words - h) / (uint32_t)kCoopWords : 0u;
}

__device__ __forceinline__ mcd::Affine affine_steps(const mcd::Affine* tab, uint64_t k) {
  mcd::Affine acc{1ull, 0ull};
  while (k) {
    const int j = __ffsll((long long)k) - 1;
    acc = mcd::compose(tab[j], acc);
    k &= k - 1;
  }
  return acc;
}

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  return ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(a);
}
__device__ __forceinline__ float lo_of(unsigned long long w) { return __uint_as_float((uint32_t)w); }
__device__ __forceinline__ float hi_of(unsigned long long w) { return __uint_as_float((uint32_t)(w >> 32)); }
__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double dval(unsigned long long w) { return __longlong_as_double((long long)w); }

// A history's record: its stream, particle, ids, tally sink and the counts
// of its events in the tail.
struct CoopHist {
  unsigned long long* w;
  enum {
    kX = 0,      // stream state
    kDraws,      // draws taken
    kPos,        // fp64 x (fp32: xf, xlo)
    kDir,        // fp64 mu (fp32: muf, wf)
    kW,          // fp64 2^32 / |mu|
    kGi,         // global history index
    kEvents,     // flights flown
    kProb,       // problem index; bit 32: live
    kBase,       // tally row
    kEdges,      // edge and width tables (null: computed)
    kWidths,
    kFlights,    // counts of the tail's events
    kColl,
    kScat,
    kEnd,        // last round: events run (low half) and how the last one ended (high half)
    kSpare
  };
  __device__ __forceinline__ explicit CoopHist(unsigned long long* p) : w(p) {}
  __device__ __forceinline__ bool live() const { return (w[kProb] >> 32) != 0ull; }
  __device__ __forceinline__ const SlabDev* prob(const SlabDev* probs) const { return probs + (uint32_t)w[kProb]; }
  __device__ __forceinline__ mcs::Sink sink(bool agg) const {
    return mcs::Sink{reinterpret_cast<unsigned long long*>(w[kBase]), reinterpret_cast<const double*>(w[kEdges]),
                     reinterpret_cast<const double*>(w[kWidths]), agg};
  }
};

// The records of one history's round, six arrays of E + 1 words.
struct CoopRec {
  unsigned long long* p;  // p_e = d_e mu_e (fp32: pr and pe, the product and its error)
  unsigned long long* d;  // d_e (fp32: d_e and muf_e)
  unsigned long long* m;  // mu_e (fp32: the state of event e's distance draw)
  unsigned long long* w;  // tally weight of event e's flight
  unsigned long long* x;  // position at the start of event e
  unsigned long long* f;  // absorption test of event e
  __device__ __forceinline__ CoopRec(unsigned long long* r, uint32_t E)
      : p(r), d(r + (E + 1u)), m(r + 2u * (E + 1u)), w(r + 3u * (E + 1u)), x(r + 4u * (E + 1u)),
        f(r + 5u * (E + 1u)) {}
};

// Phase 1, on lane hl of the G lanes of a history's group: the draw-only
// values of the events e = hl, hl + G, ... <= E.
template <int M, bool F32>
__device__ __noinline__ void coop_draws(const CoopArgs* c, const mcd::Affine* tab, uint32_t hist_off,
                                        uint32_t rec_off, uint32_t E, int G, int hl) {
  extern __shared__ unsigned long long s_dyn[];
  const CoopHist H(s_dyn + hist_off);
  const CoopRec R(s_dyn + rec_off, E);
  const mcd::Lcg l = c->t.lcg;
  const SlabDev& p = *H.prob(c->probs);
  const uint64_t x0 = H.w[CoopHist::kX];
  const unsigned long long dir0 = H.w[CoopHist::kDir], w0 = H.w[CoopHist::kW];
  const mcd::Affine step3g = affine_steps(tab, 3ull * (uint64_t)G);
  uint64_t xs = mcs::skip_tab(tab, x0, 3ull * (uint64_t)hl);  // the state after 3e draws
  for (uint32_t e = (uint32_t)hl; e <= E; e += (uint32_t)G) {
    if constexpr (!F32) {
      double mu = dval(dir0), w = dval(w0);
      if (e != 0u) {
        mu = mcx::two_u_minus_1(mcd::u53<M>(xs, l.m));
        w = mcs::fix_per_mu(mu);
      }
      R.m[e] = dbits(mu);
      R.w[e] = dbits(w);
      if (e < E) {
        const uint64_t sd = mcd::lcg_step(xs, l.g, l.c);
        const double d = __dmul_rn(-mclog::log1m_n(mcd::u53<M>(sd, l.m)), p.inv_st);
        R.d[e] = dbits(d);
        R.p[e] = dbits(__dmul_rn(d, mu));
        R.f[e] = mcd::u53<M>(mcd::lcg_step(sd, l.g, l.c), l.m) < p.p_abs_n ? 1ull : 0ull;
      }
    } else {
      float muf = lo_of(dir0), wf = hi_of(dir0);
      if (e != 0u) {
        muf = mcs::mu_f32(mcd::u53<M>(xs, l.m));
        wf = muf != 0.0f ? __frcp_rn(fabsf(muf)) : 0.0f;
      }
      R.w[e] = pack2(wf, 0.0f);
      float d = 0.0f;
      if (e < E) {
        const uint64_t sd = mcd::lcg_step(xs, l.g, l.c);
        d = mcs::flight_f32(mcd::u01<M>(sd, l.m)) * p.inv_st_f;
        const float pr = __fmul_rn(d, muf);
        R.p[e] = pack2(pr, __fmaf_rn(d, muf, -pr));
        R.m[e] = sd;
        R.f[e] = mcd::u53<M>(mcd::lcg_step(sd, l.g, l.c), l.m) < p.p_abs_n ? 1ull : 0ull;
      }
      R.d[e] = pack2(d, muf);
    }
    xs = mcd::apply(step3g, xs);
  }
}

// Phase 2, on one lane: the chain of positions through the round's events,
// until the round ends (kContinue), an event would pass the cap (-1), or the
// history leaks or is absorbed.  Then the history's record moves on by the
// events run, and a history that ended is counted and written out.
template <int M, bool F32>
__device__ __noinline__ void coop_walk(const CoopArgs* c, const mcd::Affine* tab, uint32_t hist_off,
                                       uint32_t rec_off, uint32_t E) {
  extern __shared__ unsigned long long s_dyn[];
  const CoopHist H(s_dyn + hist_off);
  const CoopRec R(s_dyn + rec_off, E);
  const SlabDev* P = H.prob(c->probs);
  const SlabDev p = *P;
  const uint64_t events = H.w[CoopHist::kEvents];
  const uint64_t left = c->t.event_cap - events;  // events never pass the cap
  const uint32_t ok = left < E ? (uint32_t)left : E;
  int out = mcs::kContinue;
  uint32_t e = 0;
  // Four events at a time while none of them can end the history (no
  // leak, no absorption, no cap, and in fp32 no guard band): the chain of
  // additions runs back to back and one branch takes the four.  Otherwise
  // one event at a time, with the same operations.
  if constexpr (!F32) {
    double x = dval(H.w[CoopHist::kPos]);
    R.x[0] = dbits(x);
    for (;;) {
      if (e + 4u <= ok) {
        const double p0 = dval(R.p[e]), p1 = dval(R.p[e + 1u]), p2 = dval(R.p[e + 2u]), p3 = dval(R.p[e + 3u]);
        const long long m0 = (long long)R.m[e], m1 = (long long)R.m[e + 1u], m2 = (long long)R.m[e + 2u],
                        m3 = (long long)R.m[e + 3u];
        const unsigned long long a = R.f[e] | R.f[e + 1u] | R.f[e + 2u] | R.f[e + 3u];
        const double x1 = __dadd_rn(x, p0), x2 = __dadd_rn(x1, p1), x3 = __dadd_rn(x2, p2), x4 = __dadd_rn(x3, p3);
        if (!(a | mcs::leaves64(p, m0, x1) | mcs::leaves64(p, m1, x2) | mcs::leaves64(p, m2, x3) |
              mcs::leaves64(p, m3, x4))) {
          R.x[e + 1u] = dbits(x1);
          R.x[e + 2u] = dbits(x2);
          R.x[e + 3u] = dbits(x3);
          R.x[e + 4u] = dbits(x4);
          x = x4;
          e += 4u;
          continue;
        }
      }
      if (e == E) break;
      if (e == ok) { out = -1; break; }
      double xn;
      const int f = mcs::advance64(p, x, dval(R.m[e]), dval(R.p[e]), xn);
      if (f != mcs::kCollide) { out = f; ++e; break; }
      x = xn;
      R.x[e + 1u] = dbits(x);
      if (R.f[e]) { out = mcs::kAbsorbed; ++e; break; }
      ++e;
    }
    H.w[CoopHist::kPos] = dbits(x);
    if (out == mcs::kContinue) { H.w[CoopHist::kDir] = R.m[E]; H.w[CoopHist::kW] = R.w[E]; }
  } else {
    const unsigned long long pos = H.w[CoopHist::kPos];
    float xf = lo_of(pos), xlo = hi_of(pos);
    R.x[0] = pos;
    const uint32_t m = c->t.lcg.m;
    for (;;) {
      if (e + 4u <= ok) {
        const unsigned long long q0 = R.p[e], q1 = R.p[e + 1u], q2 = R.p[e + 2u], q3 = R.p[e + 3u];
        const float u0 = hi_of(R.d[e]), u1 = hi_of(R.d[e + 1u]), u2 = hi_of(R.d[e + 2u]), u3 = hi_of(R.d[e + 3u]);
        const unsigned long long a = R.f[e] | R.f[e + 1u] | R.f[e + 2u] | R.f[e + 3u];
        float h1, l1, h2, l2, h3, l3, h4, l4;
        mcs::pair_step(xf, xlo, lo_of(q0), hi_of(q0), h1, l1);
        mcs::pair_step(h1, l1, lo_of(q1), hi_of(q1), h2, l2);
        mcs::pair_step(h2, l2, lo_of(q2), hi_of(q2), h3, l3);
        mcs::pair_step(h3, l3, lo_of(q3), hi_of(q3), h4, l4);
        if (a == 0ull && mcs::plain_collision32(p, u0, h1, l1) && mcs::plain_collision32(p, u1, h2, l2) &&
            mcs::plain_collision32(p, u2, h3, l3) && mcs::plain_collision32(p, u3, h4, l4)) {
          R.x[e + 1u] = pack2(h1, l1);
          R.x[e + 2u] = pack2(h2, l2);
          R.x[e + 3u] = pack2(h3, l3);
          R.x[e + 4u] = pack2(h4, l4);
          xf = h4;
          xlo = l4;
          e += 4u;
          continue;
        }
      }
      if (e == E) break;
      if (e == ok) { out = -1; break; }
      const unsigned long long pc = R.p[e];
      float xn, xnlo;
      const int f = mcs::advance32(p, xf, xlo, hi_of(R.d[e]), lo_of(pc), hi_of(pc),
                                   [&] { return mcd::u01<M>(R.m[e], m); }, xn, xnlo);
      if (f != mcs::kCollide) { out = f; ++e; break; }
      xf = xn;
      xlo = xnlo;
      R.x[e + 1u] = pack2(xf, xlo);
      if (R.f[e]) { out = mcs::kAbsorbed; ++e; break; }
      ++e;
    }
    H.w[CoopHist::kPos] = pack2(xf, xlo);
    if (out == mcs::kContinue) H.w[CoopHist::kDir] = pack2(hi_of(R.d[E]), lo_of(R.w[E]));
  }
  // every event run is a flight; a collision unless it leaked; then an
  // absorption or a scattering
  const bool leaked = out == mcs::kLeakLo || out == mcs::kLeakHi;
  H.w[CoopHist::kEvents] = events + e;
  H.w[CoopHist::kFlights] += e;
  H.w[CoopHist::kColl] += e - (leaked ? 1u : 0u);
  H.w[CoopHist::kScat] += e - (leaked || out == mcs::kAbsorbed ? 1u : 0u);
  H.w[CoopHist::kEnd] = (unsigned long long)e | ((unsigned long long)(uint32_t)out << 32);
  // draws taken: three per completed event, one for a leaking flight, two
  // for an absorbed one, none for a capped event
  const uint64_t used = out == mcs::kContinue ? 3ull * E
                      : out == -1 ? 3ull * e
                      : out == mcs::kAbsorbed ? 3ull * e - 1ull : 3ull * e - 2ull;
  const uint64_t x = mcs::skip_tab(tab, H.w[CoopHist::kX], used);
  const uint64_t draws = H.w[CoopHist::kDraws] + used;
  H.w[CoopHist::kX] = x;
  H.w[CoopHist::kDraws] = draws;
  if (out == mcs::kContinue) return;
  // the history's end: its counts as the one-lane path would flush them
  const uint32_t pi = (uint32_t)H.w[CoopHist::kProb];
  unsigned long long* cnt = c->t.counts + (size_t)pi * MC_NCOUNT;
  atomicAdd(cnt + MC_C_FLIGHTS, H.w[CoopHist::kFlights]);
  if (H.w[CoopHist::kColl]) atomicAdd(cnt + MC_C_COLLISIONS, H.w[CoopHist::kColl]);
  if (H.w[CoopHist::kScat]) atomicAdd(cnt + MC_C_SCATTERS, H.w[CoopHist::kScat]);
  if (out == mcs::kAbsorbed) atomicAdd(cnt + MC_C_ABSORPTIONS, 1ull);
  else if (out == mcs::kLeakLo) atomicAdd(cnt + MC_C_LEAK_LO, 1ull);
  else if (out == mcs::kLeakHi) atomicAdd(cnt + MC_C_LEAK_HI, 1ull);
  else atomicAdd(cnt + MC_C_CAPPED, 1ull);
  atomicAdd(cnt + MC_C_DRAWS, draws);
  atomicMax(cnt + MC_C_MAX_DRAWS, draws);
  if (p.stride_q != 0 && draws > p.stride_q) {
    atomicAdd(cnt + MC_C_EXCEED_HIST, 1ull);
    atomicAdd(cnt + MC_C_EXCEED_DRAWS, draws - p.stride_q);
  }
  const uint64_t gi = H.w[CoopHist::kGi];
  if (c->t.hist_state) c->t.hist_state[gi] = x & c->t.lcg.mask;
  if (c->t.hist_draws) c->t.hist_draws[gi] = draws;
  H.w[CoopHist::kProb] = pi;  // no longer live
}

// Phase 3, on lane hl of the group: the tally contributions of the round's
// events e = hl, hl + G, ... of those the history ran, with warp-aggregated
// atomics whatever the launch's setting (the bits are the same either way):
// the lanes of a group tally consecutive events of one history, mostly in
// the same bins.
template <bool F32>
__device__ __noinline__ void coop_tally(const CoopArgs* c, uint32_t hist_off, uint32_t rec_off, uint32_t E, int G,
                                        int hl) {
  extern __shared__ unsigned long long s_dyn[];
  const CoopHist H(s_dyn + hist_off);
  const CoopRec R(s_dyn + rec_off, E);
  const SlabDev& p = *H.prob(c->probs);
  const mcs::Sink sk = H.sink(true);
  const unsigned long long end = H.w[CoopHist::kEnd];
  const int nev = (int)(uint32_t)end, out = (int)(uint32_t)(end >> 32);
  for (int e = hl; e < nev; e += G) {
    const int f = (e == nev - 1 && (out == mcs::kLeakLo || out == mcs::kLeakHi)) ? out : mcs::kCollide;
    if constexpr (!F32) {
      const double xe = dval(R.x[e]);
      const double xn = f == mcs::kCollide ? dval(R.x[e + 1]) : 0.0;
      mcs::tally64(p, xe, xn, dval(R.m[e]), dval(R.d[e]), dval(R.w[e]), f, sk);
    } else {
      const unsigned long long xa = R.x[e];
      const unsigned long long xb = f == mcs::kCollide ? R.x[e + 1] : 0ull;
      const unsigned long long dw = R.d[e];
      mcs::tally32(p, lo_of(xa), hi_of(xa), lo_of(xb), hi_of(xb), hi_of(dw), lo_of(dw), lo_of(R.w[e]), f, sk);
    }
  }
}

// The rounds, warp-uniform, over the n_in history records at area_off.
template <int M, bool F32>
__device__ __noinline__ void coop_tail(const CoopArgs* c, const mcd::Affine* tab, uint32_t area_off,
                                       uint32_t slots, int n_in) {
  extern __shared__ unsigned long long s_dyn[];
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t rec_base = area_off + (uint32_t)(kCoopMax * kCoopHistWords);
  for (;;) {
    __syncwarp();
    unsigned live = 0u;
    for (int h = 0; h < n_in; ++h)
      if (CoopHist(s_dyn + area_off + (uint32_t)h * kCoopHistWords).live()) live |= 1u << h;
    if (live == 0u) break;
    const int nl = __popc(live);
    const int kp = coop_groups(nl);
    const int G = 32 / kp;
    const int grp = (int)lane / G, hl = (int)lane % G;
    unsigned m = live;
    for (int i = 0; i < grp && m != 0u; ++i) m &= m - 1u;
    const int h = (grp < nl && m != 0u) ? __ffs(m) - 1 : -1;
    const uint32_t E = coop_events(slots, kp);
    const uint32_t hist_off = area_off + (uint32_t)(h < 0 ? 0 : h) * kCoopHistWords;
    const uint32_t rec_off = rec_base + (uint32_t)grp * (E + 1u) * kCoopWords;
    __syncwarp();
    if (h >= 0) coop_draws<M, F32>(c, tab, hist_off, rec_off, E, G, hl);
    __syncwarp();
    if (h >= 0 && hl == 0) coop_walk<M, F32>(c, tab, hist_off, rec_off, E);
    __syncwarp();
    if (h >= 0) coop_tally<F32>(c, hist_off, rec_off, E, G, hl);
  }
}

template <int M, bool F32, bool SMEM, bool AGG>
__device__ __forceinline__ void slab_history_body(const RunArgs& a) {
  extern __shared__ unsigned long long s_tally[];
  __shared__ mcd::Affine tab[64];
  if (threadIdx.x == 0) {
    mcd::Affine sq{a.lcg.g, a.lcg.c};
    for (int j = 0; j < 64; ++j) { tab[j] = sq; sq = mcd::compose(sq, sq); }
  }
  if constexpr (SMEM) {
    for (uint32_t s = threadIdx.x; s < a.smem_slots; s += blockDim.x) s_tally[s] = 0ull;
  }
  double* s_edges = a.smem_edges ? reinterpret_cast<double*>(s_tally + (SMEM ? a.smem_slots : 0u)) : nullptr;
  double* s_widths = s_edges ? s_edges + a.smem_edges : nullptr;  // n_bins widths after the edges
  // the particle pool after the tally and the edge tables
  unsigned long long* s_pool = s_tally + (SMEM ? a.smem_slots : 0u) + 2u * a.smem_edges;
  __shared__ PoolCtl ctl;
  if (threadIdx.x == 0) {
    ctl.lock = 0;
    ctl.n = 0;
    ctl.active = (int)(blockDim.x >> 5);
    ctl.pad = 0;
  }
  if (s_edges) {
    const SlabDev& p0 = a.probs[0];
    for (uint32_t j = threadIdx.x; j + 1 < a.smem_edges; j += blockDim.x)
      s_widths[j] = __dsub_rn(mcs::slab_edge(p0, (int)j + 1), mcs::slab_edge(p0, (int)j));
  }
  if (s_edges) {
    const SlabDev& p0 = a.probs[0];
    for (uint32_t j = threadIdx.x; j < a.smem_edges; j += blockDim.x) s_edges[j] = mcs::slab_edge(p0, (int)j);
  }
  __syncthreads();

  const unsigned kFull = 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt_mask = (1u << lane) - 1u;
  const mcd::Lcg l = a.lcg;

  uint64_t pool_next = 0, pool_end = 0;
  bool more = true;
  bool alive = false;
  mcs::LaneCounts lc;
  lc.prob = -1;
  lc.clear();

  const SlabDev* P = a.probs;
  mcs::Rng<M> r{0ull, 0ull};
  mcs::SlabParticle q{};
  mcs::Sink sink{nullptr, s_edges, s_widths, AGG};
  uint64_t gi = 0, events = 0;
  int coop_n = 0;  // histories handed to the cooperative tail (warp-uniform)

  for (;;) {
    unsigned dead = __ballot_sync(kFull, !alive);
    while (dead != 0u && more) {
      if (pool_next >= pool_end) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.ticket, (unsigned long long)a.chunk);
        base = __shfl_sync(kFull, base, 0);
        if (base >= a.total) { more = false; break; }
        pool_next = base;
        pool_end = min((uint64_t)base + (uint64_t)a.chunk, (uint64_t)a.total);
      }
      const uint64_t avail = pool_end - pool_next;
      const unsigned rank = __popc(dead & lt_mask);
      if (!alive && rank < avail) {
        uint32_t pi;
        mcs::ticket_history(a.probs, a.nprob, a.range_begin, a.order, pool_next + rank, pi, gi);
        if ((int)pi != lc.prob) { lc.flush(a.counts); lc.prob = (int)pi; }
        P = a.probs + pi;
        const uint64_t id = gi - P->hist_begin;
        const uint64_t batch = mcs::batch_of(id, P->n_hist, P->n_batches);
        sink.base = (SMEM ? s_tally : a.tally) + P->tally_offset + batch * P->n_bins;
        if (a.tables) {
          sink.edges = a.tables + P->tab_off;
          sink.widths = sink.edges + P->n_bins + 1;
        }
        r.x = mcs::slab_seed(*P, id, tab, l.mask);
        r.draws = 0;
        mcs::slab_source<M, F32>(*P, r, l, q);
        events = 0;
        ++lc.src;
        alive = true;
      }
      pool_next += min((uint64_t)__popc(dead), avail);
      dead = __ballot_sync(kFull, !alive);
    }
    if (!more && a.pool_cap != 0u) {
      // ticket exhausted: take particles from the block's pool into dead
      // lanes, hand this warp's few over, or leave
      // the pool's count and active warps as lane 0 reads them: every branch
      // below must be taken by the whole warp (full-mask shuffles inside)
      volatile PoolCtl& vc = ctl;
      const int hint_n = __shfl_sync(kFull, lane == 0 ? vc.n : 0, 0);
      const int hint_active = __shfl_sync(kFull, lane == 0 ? vc.active : 0, 0);
      if (dead != 0u && hint_n > 0) {
        int k = 0, n = 0, ok = 0;
        if (lane == 0) {
          ok = pool_lock(&ctl.lock, a.lock_attempts);
          if (ok) {
            n = vc.n;
            k = min(n, __popc(dead));
            vc.n = n - k;
          }
        }
        k = __shfl_sync(kFull, k, 0);
        n = __shfl_sync(kFull, n, 0);
        if (k < 0 || n > (int)a.pool_cap || k > n) k = 0;  // never outside the pool
        __syncwarp();
        const unsigned rank = __popc(dead & lt_mask);
        if (!alive && (int)rank < k) {
          const uint32_t pi = pool_get<M>(s_pool + (size_t)(n - k + (int)rank) * kPoolWords, r, q, gi, events);
          if ((int)pi != lc.prob) { lc.flush(a.counts); lc.prob = (int)pi; }
          P = a.probs + pi;
          const uint64_t id = gi - P->hist_begin;
          sink.base = (SMEM ? s_tally : a.tally) + P->tally_offset + mcs::batch_of(id, P->n_hist, P->n_batches) * P->n_bins;
          if (a.tables) {
            sink.edges = a.tables + P->tab_off;
            sink.widths = sink.edges + P->n_bins + 1;
          }
          alive = true;
        }
        __syncwarp();
        if (lane == 0 && ok) pool_unlock(&ctl.lock);
        dead = __ballot_sync(kFull, !alive);
      }
      const unsigned live = ~dead;
      const int nlive = __popc(live);
      if (nlive != 0 && nlive <= kCoopMax && hint_active == 1 && hint_n == 0 &&
          coop_events(a.coop_slots, coop_groups(nlive)) >= kCoopMinEvents) {
        // the block's last warp with a few long histories: confirm under the
        // lock that no warp is left to fill the pool, then finish them
        // together
        int ok = 0;
        if (lane == 0 && pool_lock(&ctl.lock, a.lock_attempts)) {
          ok = (vc.n == 0 && vc.active == 1) ? 1 : 0;
          pool_unlock(&ctl.lock);
        }
        if (__shfl_sync(kFull, ok, 0)) {
          lc.flush_warp(a.counts);
          if (alive) {
            CoopHist H(s_pool + (size_t)__popc(live & lt_mask) * kCoopHistWords);
            H.w[CoopHist::kX] = r.x;
            H.w[CoopHist::kDraws] = r.draws;
            H.w[CoopHist::kPos] = F32 ? pack2(q.xf, q.xlo) : dbits(q.x);
            H.w[CoopHist::kDir] = F32 ? pack2(q.muf, q.wf) : dbits(q.mu);
            H.w[CoopHist::kW] = dbits(q.w_mu);
            H.w[CoopHist::kGi] = gi;
            H.w[CoopHist::kEvents] = events;
            H.w[CoopHist::kProb] = (uint64_t)(uint32_t)(P - a.probs) | (1ull << 32);
            H.w[CoopHist::kBase] = reinterpret_cast<unsigned long long>(sink.base);
            H.w[CoopHist::kEdges] = reinterpret_cast<unsigned long long>(sink.edges);
            H.w[CoopHist::kWidths] = reinterpret_cast<unsigned long long>(sink.widths);
            H.w[CoopHist::kFlights] = H.w[CoopHist::kColl] = H.w[CoopHist::kScat] = 0ull;
          }
          coop_n = nlive;
          alive = false;
          break;
        }
      }
      if (nlive == 0 || (nlive <= (int)a.donate_max && hint_active > 1 && hint_n + nlive <= (int)a.pool_cap)) {
        int go = 0, n = 0;
        if (lane == 0) {
          if (pool_lock(&ctl.lock, a.lock_attempts)) {
            n = vc.n;
            if (nlive == 0 ? n == 0 : (vc.active > 1 && n + nlive <= (int)a.pool_cap)) {
              vc.n = n + nlive;
              vc.active = vc.active - 1;
              go = 1;
            }
            if (!go || nlive == 0) pool_unlock(&ctl.lock);
          } else if (nlive == 0) {
            // cannot see the pool: leave, counting what may be stranded
            atomicAdd(a.counts + MC_C_DROPPED, (unsigned long long)max(vc.n, 0));
            go = 1;
          }
        }
        go = __shfl_sync(kFull, go, 0);
        n = __shfl_sync(kFull, n, 0);
        if (go) {
          if (nlive != 0) {
            const uint32_t slot = (uint32_t)n + (uint32_t)__popc(live & lt_mask);
            if (alive && slot < a.pool_cap)  // always, by the count taken under the lock
              pool_put<M>(s_pool + (size_t)slot * kPoolWords, r, q, gi, events, (uint32_t)(P - a.probs));
            else if (alive)
              atomicAdd(a.counts + MC_C_DROPPED, 1ull);
            __syncwarp();
            if (lane == 0) pool_unlock(&ctl.lock);
            alive = false;
          }
          break;
        }
        if (nlive == 0) continue;  // the pool holds particles: take them on the next pass
      }
    } else if (__ballot_sync(kFull, alive) == 0u) {
      break;
    }
    if (alive) {
      int outcome;
      if (events == a.event_cap) {
        ++lc.capped;
        outcome = -1;
      } else {
        ++events;
        ++lc.flights;
        outcome = mcs::slab_event<M, F32>(*P, r, l, q, sink, lc.coll, lc.scat);
        if (outcome == mcs::kAbsorbed) ++lc.absn;
        else if (outcome == mcs::kLeakLo) ++lc.llo;
        else if (outcome == mcs::kLeakHi) ++lc.lhi;
      }
      if (outcome != mcs::kContinue) {
        end_history<M>(TailArgs{a.hist_state, a.hist_draws, a.counts, a.lcg, a.event_cap}, r, P, gi, lc);
        alive = false;
      }
    }
  }
  if (coop_n != 0) {
    // the arguments through shared memory too: a call with them by value
    // would put them on the stack of the whole kernel
    __shared__ CoopArgs s_coop;
    if (lane == 0) s_coop = CoopArgs{TailArgs{a.hist_state, a.hist_draws, a.counts, a.lcg, a.event_cap}, a.probs};
    __syncwarp();
    coop_tail<M, F32>(&s_coop, tab, (uint32_t)(s_pool - s_tally), a.coop_slots, coop_n);
  }
  lc.flush_warp(a.counts);

  if constexpr (SMEM) {
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < a.smem_slots; s += blockDim.x) {
      const unsigned long long v = s_tally[s];
      if (v != 0ull) atomicAdd(a.tally + s, v);
    }
  }
}

// The kernel in two register budgets.  The fp32 flight fits 64 registers
// (four blocks of 256 per SM); the fp64 flight spills there, and runs faster
// with 80 and three blocks per SM (slab_long 240 -> 215 ms, batched 23.4 ->
// 20.6 ms; the fp32 kernel at 80 measured batched 18.0 -> 19.8 ms).  Both
// accept blocks of up to 512 threads.
template <int M, bool F32, bool SMEM, bool AGG>
__global__ void __launch_bounds__(512, 2) slab_history_kernel_f32(const RunArgs a) {
  slab_history_body<M, F32, SMEM, AGG>(a);
}
template <int M, bool F32, bool SMEM, bool AGG>
__global__ void __maxnreg__(80) slab_history_kernel_f64(const RunArgs a) {
  slab_history_body<M, F32, SMEM, AGG>(a);
}

template <int M, bool F32, bool SMEM, bool AGG>
auto history_kernel_of() {
  if constexpr (F32) return slab_history_kernel_f32<M, F32, SMEM, AGG>;
  else return slab_history_kernel_f64<M, F32, SMEM, AGG>;
}

template <int M, bool F32, bool SMEM, bool AGG>
int launch_history(const RunArgs& a0, int block, int blocks_per_sm, int num_sms, cudaStream_t s) {
  auto k = history_kernel_of<M, F32, SMEM, AGG>();
  RunArgs a = a0;
  // Static shared memory of this instantiation (read once) and the device's
  // opt-in limit: what does not fit beside them is given up, the compaction
  // pool first and then the edge tables (both only save time).
  static size_t static_smem = ~(size_t)0;
  if (static_smem == ~(size_t)0) {
    cudaFuncAttributes fa{};
    const int st = mci::cuda_status(cudaFuncGetAttributes(&fa, k), "cudaFuncGetAttributes(slab_history_kernel)");
    if (st != MC_OK) return st;
    static_smem = fa.sharedSizeBytes;
  }
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the pool's memory, which the cooperative tail reuses: at least
  // kCoopAreaWords when there is a pool
  auto pool_words = [&a]() {
    return a.pool_cap ? std::max<size_t>((size_t)a.pool_cap * kPoolWords, kCoopAreaWords) : (size_t)0;
  };
  auto dynamic_smem = [&a, &pool_words]() {
    return (SMEM ? (size_t)a.smem_slots * 8u : 0u) + (size_t)a.smem_edges * 16u +  // edges + widths
           pool_words() * 8u;
  };
  if (static_smem + dynamic_smem() > (size_t)optin) a.pool_cap = 0;
  if (static_smem + dynamic_smem() > (size_t)optin) a.smem_edges = 0;
  a.coop_slots = coop_slots_of((uint32_t)pool_words());
  const size_t smem = dynamic_smem();
  if (static_smem + smem > (size_t)optin) {
    mci::set_error("slab_history_kernel: %u tally slots do not fit in shared memory", a.smem_slots);
    return MC_ERR_ARG;
  }
  if (static_smem + smem > 48u * 1024u) {
    int st = mci::cuda_status(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                              "cudaFuncSetAttribute(slab_history_kernel)");
    if (st != MC_OK) return st;
  }
  int per_sm = blocks_per_sm;
  if (per_sm <= 0) {
    int st = mci::cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem),
                              "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (st != MC_OK) return st;
    if (per_sm < 1) per_sm = 1;
  }
  // Enough warps for every chunk, never more than fill the GPU.
  const uint64_t warps_needed = (a.total + a.chunk - 1) / a.chunk;
  const uint64_t blocks_needed = (warps_needed * 32 + block - 1) / block;
  const uint64_t full = (uint64_t)num_sms * (uint64_t)per_sm;
  const int grid = (int)std::max<uint64_t>(1, std::min(full, blocks_needed));
  k<<<grid, block, smem, s>>>(a);
  return mci::cuda_status(cudaGetLastError(), "slab_history_kernel launch");
}

template <int M, bool AGG>
int launch_history_m(const RunArgs& a, bool f32, int block, int bps, int sms, cudaStream_t s) {
  const bool smem = a.smem_slots != 0;
  if (f32) return smem ? launch_history<M, true, true, AGG>(a, block, bps, sms, s)
                       : launch_history<M, true, false, AGG>(a, block, bps, sms, s);
  return smem ? launch_history<M, false, true, AGG>(a, block, bps, sms, s)
              : launch_history<M, false, false, AGG>(a, block, bps, sms, s);
}

}  // namespace

namespace mci {

size_t slab_dev_size() { return sizeof(SlabDev); }

void slab_fill_host(const mc_problem* src, uint32_t n, void* dst) {
  SlabDev* d = static_cast<SlabDev*>(dst);
  uint64_t off = 0;
  for (uint32_t i = 0; i < n; ++i) {
    SlabDev q;
    std::memset(&q, 0, sizeof q);
    q.L = src[i].L;
    q.sigma_t = src[i].sigma_t;
    q.c = src[i].c;
    q.n_hist = src[i].n_histories;
    q.seed = src[i].seed;
    q.stride_q = src[i].stride_q;
    q.id_offset = src[i].id_offset;
    q.key = src[i].key;
    q.tally_offset = src[i].tally_offset;
    q.n_bins = src[i].n_bins;
    q.n_batches = src[i].n_batches;
    q.source = src[i].source;
    q.seeding = src[i].seeding;
    q.tab_off = off;
    off += 2ull * q.n_bins + 1ull;
    d[i] = q;
  }
}

int slab_prep(void* d_probs, uint32_t n, cudaStream_t s, void* d_tables, void* d_order) {
  uint32_t* order = d_order && n >= 2 && n <= kMaxOrderedProblems ? static_cast<uint32_t*>(d_order) : nullptr;
  uint64_t* begin = order ? reinterpret_cast<uint64_t*>(order + ((n + 1u) & ~1u)) : nullptr;
  slab_prep_kernel<<<1, 256, 0, s>>>(static_cast<SlabDev*>(d_probs), n, order, begin);
  int st = cuda_status(cudaGetLastError(), "slab_prep_kernel launch");
  if (st != MC_OK || !d_tables) return st;
  slab_tables_kernel<<<std::min<uint32_t>(n, 1024u), 64, 0, s>>>(static_cast<const SlabDev*>(d_probs), n,
                                                                   static_cast<double*>(d_tables));
  return cuda_status(cudaGetLastError(), "slab_tables_kernel launch");
}

uint64_t slab_table_doubles(const mc_problem* src, uint32_t n) {
  uint64_t t = 0;
  for (uint32_t i = 0; i < n; ++i) t += 2ull * src[i].n_bins + 1ull;
  return t;
}

int slab_history_launch(const SlabLaunch& L, cudaStream_t s) {
  RunArgs a{};
  a.probs = static_cast<const SlabDev*>(L.d_probs);
  a.nprob = L.n_problems;
  a.chunk = L.chunk;
  a.range_begin = L.range_begin;
  a.total = L.total;
  a.ticket = L.d_ticket;
  a.tally = reinterpret_cast<unsigned long long*>(L.tally->d_bins);
  a.counts = reinterpret_cast<unsigned long long*>(L.tally->d_counts);
  a.hist_state = L.tally->d_hist_state;
  a.hist_draws = L.tally->d_hist_draws;
  a.lcg = mcd::Lcg{L.lcg.g, L.lcg.c, mcd::mask_of(L.lcg.m), L.lcg.m};
  a.event_cap = L.event_cap;
  a.smem_slots = L.smem_slots;
  a.smem_edges = 0;
  if (L.n_problems == 1) {
    // one problem: its bin edges from a shared-memory table (the problem's
    // bin count comes from the host copy through the launch descriptor)
    if (L.single_n_bins + 1 <= 4096) a.smem_edges = L.single_n_bins + 1;
  }
  // otherwise each problem's tables in global memory, where staged
  a.tables = a.smem_edges ? nullptr : static_cast<const double*>(L.d_tables);
  // compaction: a warp with at most 12 live lanes hands them over; the pool
  // holds what every other warp of the block could hand over
  a.donate_max = 12;
  a.pool_cap = L.block >= 64 ? (uint32_t)((L.block >> 5) - 1) * a.donate_max : 0u;
  a.lock_attempts = L.pool_lock_attempts;
  a.order = mcs::Order{L.d_order, L.d_order_begin};
  if (L.tally_agg) {
    if (L.lcg.m == 63) return launch_history_m<63, true>(a, L.f32, L.block, L.blocks_per_sm, L.num_sms, s);
    return launch_history_m<0, true>(a, L.f32, L.block, L.blocks_per_sm, L.num_sms, s);
  }
  if (L.lcg.m == 63) return launch_history_m<63, false>(a, L.f32, L.block, L.blocks_per_sm, L.num_sms, s);
  return launch_history_m<0, false>(a, L.f32, L.block, L.blocks_per_sm, L.num_sms, s);
}

}  // namespace mci

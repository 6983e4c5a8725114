// slab.cuh -- device view of a slab problem and the per-particle physics
// shared by the history-based and the event-based slab schedules.
//
// Both schedules call the same functions below for every draw, flight,
// collision and tally contribution, so they make the same int64 tally
// contributions; int64 addition is associative, so the totals are
// bit-identical whatever the order of the additions.
//
// fp64 path: every operation is the one the transport definition names,
// rounded once (this file is compiled with --fmad=false, so no a*b+c is
// contracted).  fp32 path: flight length and geometry in fp32, with an fp64
// recomputation of the leak/collide decision when the fp32 end point lands
// within a guard band of a slab face; uniforms, absorption tests and the
// fixed-point scaling of tally contributions stay exact (fp64 or integer).
#pragma once
#include <cstdint>

#include "../../include/mc.h"
#include "mc_device.cuh"
#include "fp_exact.cuh"
#include "mc_log.cuh"

namespace mcs {

struct SlabDev {
  double L, sigma_t, c;
  uint64_t n_hist, seed, stride_q, id_offset, key, tally_offset;
  uint32_t n_bins, n_batches, source, seeding;
  // derived on the device by the prep kernel
  double h;             // bin width L / n_bins
  double inv_h;         // n_bins / L: candidate-bin lookup only
  uint32_t ih_q;        // inv_h as ih_q 2^-ih_s (the lookup on the integer pipes)
  int ih_s;
  double inv_st;        // 1 / sigma_t
  double p_abs;         // 1 - c
  uint64_t p_abs_n;     // ceil((1 - c) 2^53): u < 1 - c  <=>  n < p_abs_n for u = n 2^-53
  float guard_f;        // fp32 path: half-width of the fp64 guard band at a face
  float L_f, h_f, inv_h_f, inv_st_f;
  uint64_t seed_hash;   // hash seeding: seed half of hash(., s) or of hash(., hash(key, s))
  uint64_t hist_begin;  // global index of local history 0
  uint64_t tab_off;     // its edge table (n_bins + 1) and width table (n_bins) in the table
                        // area after the records, in doubles (set on the host)
};

constexpr double kFix = 4294967296.0;  // 2^32: fixed-point scale of the tallies

// One LCG stream (Eq. 1) and its draw counter, held in registers.
template <int M>
struct Rng {
  uint64_t x;
  uint64_t draws;
  __device__ __forceinline__ double next(const mcd::Lcg& l) {
    x = mcd::lcg_step(x, l.g, l.c);
    ++draws;
    return mcd::u01<M>(x, l.m);
  }
  // The same draw as its integer n (u = n 2^-53), for comparisons and exact
  // integer arithmetic on u.
  __device__ __forceinline__ uint64_t next_n(const mcd::Lcg& l) {
    x = mcd::lcg_step(x, l.g, l.c);
    ++draws;
    return mcd::u53<M>(x, l.m);
  }
};

// The state k steps after x through a table of the maps of 2^j steps.
__device__ __forceinline__ uint64_t skip_tab(const mcd::Affine* tab, uint64_t x, uint64_t k) {
  while (k) {
    const int j = __ffsll((long long)k) - 1;
    x = mcd::apply(tab[j], x);
    k &= k - 1;
  }
  return x;
}

// Seed of local history `id` (Eqs. 2-4): hash(id, s), hash(id, hash(key, s))
// or X_{Q * (id_offset + id)}.
__device__ __forceinline__ uint64_t slab_seed(const SlabDev& p, uint64_t id, const mcd::Affine* tab,
                                              uint64_t mask) {
  if (p.seeding == MC_SEED_STRIDE) return skip_tab(tab, p.seed, p.stride_q * (p.id_offset + id)) & mask;
  return mcd::hash_with(id, p.seed_hash) & mask;
}

// The processing order of a launch of several problems: problem order[k]'s
// histories take ticket positions [begin[k], begin[k + 1]) (the prep kernel
// ranks the problems by their expected flights per history, longest first,
// so that the long chains start early and do not form the launch's tail).
// An empty order (order == nullptr) takes the histories in id order from
// range_begin.  Either way history gi keeps its own stream, so the order
// changes no result.
struct Order {
  const uint32_t* order;
  const uint64_t* begin;
};

__device__ __forceinline__ uint32_t find_problem_of(const SlabDev* p, uint32_t n, uint64_t gi) {
  uint32_t lo = 0, hi = n - 1;  // largest i with hist_begin <= gi
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (p[mid].hist_begin <= gi) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Problem and global history index of ticket position t.
__device__ __forceinline__ void ticket_history(const SlabDev* p, uint32_t n, uint64_t range_begin, const Order& o,
                                               uint64_t t, uint32_t& pi, uint64_t& gi) {
  if (o.order) {
    uint32_t lo = 0, hi = n - 1;  // largest k with begin[k] <= t
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (o.begin[mid] <= t) lo = mid; else hi = mid - 1;
    }
    pi = o.order[lo];
    gi = p[pi].hist_begin + (t - o.begin[lo]);
    return;
  }
  gi = range_begin + t;
  pi = n == 1 ? 0u : find_problem_of(p, n, gi);
}

__device__ __forceinline__ uint64_t batch_of(uint64_t id, uint64_t n_hist, uint32_t n_batches) {
  // floor(id * n_batches / n_hist) without 128-bit arithmetic when it fits.
  if (id <= (~0ull) / (n_batches ? n_batches : 1)) return (id * n_batches) / n_hist;
  const unsigned __int128 t = (unsigned __int128)id * n_batches;
  return (uint64_t)(t / n_hist);
}

__device__ __forceinline__ double slab_edge(const SlabDev& p, int j) {
  if (j >= (int)p.n_bins) return p.L;
  return j < 2048 ? mcx::mul_small((uint32_t)j, p.h) : (double)j * p.h;  // RN(j h)
}

// A bin index within one of floor(x n_bins / L), x >= 0 (integer pipes).
__device__ __forceinline__ int bin_guess(const SlabDev& p, double x) {
  return (int)min(mcx::guess_floor_mul(x, p.ih_q, p.ih_s), (uint64_t)p.n_bins);
}

__device__ __forceinline__ int clamp_bin(int j, int nb) { return j < 0 ? 0 : (j >= nb ? nb - 1 : j); }

// Tally sink: shared-memory staging or direct global atomics, and an
// optional table of the bin edges e_0..e_nb (shared memory; nullptr: each
// edge is computed as j * h).
struct Sink {
  unsigned long long* base;  // this history's [bin] row (smem or global)
  const double* edges;
  const double* widths;  // with edges: widths[j] = e_{j+1} - e_j (the same fp64 difference)
  bool agg;              // warp-aggregated atomics (mcd::warp_agg_add) instead of one per lane
  __device__ __forceinline__ void add(int j, long long v) const {
    if (v == 0) return;
    if (agg) mcd::warp_agg_add(base + j, (unsigned long long)v);
    else atomicAdd(base + j, (unsigned long long)v);
  }
};

// Order of two non-negative doubles from their bit patterns (IEEE-754
// orders non-negative values like their bits read as integers): the fp64
// comparisons of the path run on the integer pipes.
__device__ __forceinline__ bool nn_lt(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}

__device__ __forceinline__ double edge_of(const SlabDev& p, const Sink& s, int j) {
  return s.edges ? s.edges[j] : slab_edge(p, j);
}

// Track length in every bin met by the segment [a, b] (0 <= a <= b <= L):
// |[a,b] & [e_j, e_{j+1}]| / |mu|, to fixed point.  w_fix = 2^32 / |mu|,
// rounded once; since scaling by 2^32 commutes with rounding,
// (hi - lo) * w_fix rounds to exactly 2^32 times the rounded
// (hi - lo) * (1/|mu|).  The walk visits only the bins the segment
// overlaps, starting from the one that holds a.
__device__ __forceinline__ void seg64(const SlabDev& p, double a, double b, double w_fix, const Sink& s) {
  const int nb = (int)p.n_bins;
  int j = clamp_bin(bin_guess(p, a), nb);
  while (j > 0 && nn_lt(a, edge_of(p, s, j))) --j;
  while (j + 1 < nb && !nn_lt(a, edge_of(p, s, j + 1))) ++j;
  if (s.widths) {
    // The same walk with the interior bins' lengths from the width table:
    // the first bin [a, min(b, e_{j+1})], the whole bins while e_{j+1} <= b,
    // the last [e_j, b]; only the ends take an fp64 difference.
    double e1 = s.edges[j + 1];
    const double hi = nn_lt(b, e1) ? b : e1;
    if (nn_lt(a, hi)) s.add(j, mcx::llrint_nonneg(__dmul_rn(__dsub_rn(hi, a), w_fix)));
    if (!nn_lt(e1, b) || j + 1 >= nb) return;
    for (++j;; ++j) {
      e1 = s.edges[j + 1];
      if (nn_lt(b, e1)) break;
      s.add(j, mcx::llrint_nonneg(__dmul_rn(s.widths[j], w_fix)));
      if (!nn_lt(e1, b) || j + 1 >= nb) return;
    }
    const double ej = s.edges[j];
    if (nn_lt(ej, b)) s.add(j, mcx::llrint_nonneg(__dmul_rn(__dsub_rn(b, ej), w_fix)));
    return;
  }
  double lo = a;
  for (;;) {
    const double e1 = edge_of(p, s, j + 1);
    const double hi = nn_lt(b, e1) ? b : e1;
    if (nn_lt(lo, hi)) s.add(j, mcx::llrint_nonneg(__dmul_rn(__dsub_rn(hi, lo), w_fix)));
    if (!nn_lt(e1, b) || j + 1 >= nb) break;
    lo = e1;
    ++j;
  }
}

// mu == 0: the whole flight d lies in the bin holding x.
__device__ __forceinline__ void point64(const SlabDev& p, double x, double d, const Sink& s) {
  const int nb = (int)p.n_bins;
  int j = clamp_bin(bin_guess(p, x), nb);
  while (j > 0 && nn_lt(x, slab_edge(p, j))) --j;
  while (j + 1 < nb && !nn_lt(x, slab_edge(p, j + 1))) ++j;
  s.add(j, mcx::fix32_nonneg(d));
}

// Exact llrint((double)v * 2^32) for a finite float v >= 0, in integer
// arithmetic (scaling by 2^32 is exact; only values below 2^-9 need a
// rounding of the shifted-out bits, done half-to-even).
__device__ __forceinline__ long long fix32_from_float(float v) {
  const uint32_t b = __float_as_uint(v);
  const int e = (int)(b >> 23) & 0xff;
  if (e == 0) return 0;  // zero or subnormal: below 2^-126, rounds to 0 at scale 2^32
  const uint64_t mant = (uint64_t)((b & 0x7fffffu) | 0x800000u);
  const int sh = e - 127 - 23 + 32;  // value * 2^32 = mant * 2^sh
  if (sh >= 0) return (long long)(mant << sh);
  if (sh < -25) return 0;
  const int r = -sh;
  const uint64_t q = mant >> r, rem = mant & ((1ull << r) - 1ull), half = 1ull << (r - 1);
  const uint64_t up = (rem > half) || (rem == half && (q & 1ull));
  return (long long)(q + up);
}

__device__ __forceinline__ float slab_edge_f(const SlabDev& p, int j) {
  return j >= (int)p.n_bins ? p.L_f : (float)j * p.h_f;
}

// Track length of the segment [a, b] in every bin it meets, the ends given
// as pairs (ah + al, bh + bl) of the fp32 path.  Each bin's length is taken
// from the pairs, (hi_h - lo_h) + (hi_l - lo_l), so a flight whose
// displacement is far below an ulp of its position (a direction nearly
// parallel to the faces, where 1 / |mu| is large) keeps its true length
// instead of an ulp of the position times 1 / |mu|.
__device__ __forceinline__ int bin_of_pair(const SlabDev& p, float h, float l) {
  // the largest j with e_j <= h + l (fp32 edges), from the scaled guess
  const int nb = (int)p.n_bins;
  int j = clamp_bin((int)(h * p.inv_h_f), nb);
  while (j > 0) {
    const float e = slab_edge_f(p, j);
    if (h < e || (h == e && l < 0.0f)) --j; else break;
  }
  while (j + 1 < nb) {
    const float e = slab_edge_f(p, j + 1);
    if (h > e || (h == e && l >= 0.0f)) ++j; else break;
  }
  return j;
}

__device__ __forceinline__ void seg32(const SlabDev& p, float ah, float al, float bh, float bl, float w_mu,
                                      const Sink& s) {
  const int j0 = bin_of_pair(p, ah, al), j1 = bin_of_pair(p, bh, bl);
  for (int j = j0; j <= j1; ++j) {
    const float lo_e = slab_edge_f(p, j), hi_e = slab_edge_f(p, j + 1);
    // max(a, lo_e) and min(b, hi_e) as pairs (an edge's low part is zero)
    float loh = lo_e, lol = 0.0f, hih = hi_e, hil = 0.0f;
    if (ah > lo_e || (ah == lo_e && al > 0.0f)) { loh = ah; lol = al; }
    if (bh < hi_e || (bh == hi_e && bl < 0.0f)) { hih = bh; hil = bl; }
    const float len = __fadd_rn(__fsub_rn(hih, loh), __fsub_rn(hil, lol));
    if (len > 0.0f) s.add(j, fix32_from_float(__fmul_rn(len, w_mu)));
  }
}

__device__ __forceinline__ void point32(const SlabDev& p, float x, float d, const Sink& s) {
  const int nb = (int)p.n_bins;
  int j = clamp_bin((int)(x * p.inv_h_f), nb);
  while (j > 0 && x < slab_edge_f(p, j)) --j;
  while (j + 1 < nb && x >= slab_edge_f(p, j + 1)) ++j;
  s.add(j, fix32_from_float(d));
}

// Particle state of the slab physics.  fp64 path: x, mu and w_mu, which
// holds 2^32 / |mu| (0 for mu = 0); the fp32 path keeps its geometry in
// fp32: the position as an unevaluated sum xf + xlo of two floats (so that
// it does not drift from the fp64 trajectory by one rounding per flight),
// muf and wf = 1 / |muf|.
struct SlabParticle {
  double x, mu, w_mu;
  float xf, xlo, muf, wf;
};

// s + t = a + b exactly (Knuth's TwoSum; six fp32 operations, no fused
// multiply-add, so every one rounds once).
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// -ln(1 - u) in fp32 for u in [0, 1): log1pf(-u) below 1/2 (no
// cancellation for small u), else logf of 1 - u, which is exact in fp64 and
// at least 2^-53, so it rounds to a positive float and the result is finite
// (log1pf of -(float)u would meet -1 and give an infinite distance for u
// within 2^-25 of 1).
__device__ __forceinline__ float flight_f32(double u) {
  return u < 0.5 ? -log1pf(-(float)u) : -logf(__double2float_rn(__dsub_rn(1.0, u)));
}

// The fp32 direction 2u - 1 for u = n 2^-53: the exact fp64 value rounded
// once to fp32.
__device__ __forceinline__ float mu_f32(uint64_t n) { return __double2float_rn(mcx::two_u_minus_1(n)); }

// 2^32 / |mu| rounded once: 2^32 RN(1 / |mu|), the reciprocal on the
// integer pipes (fp_exact.cuh), the scaling an exponent add.
__device__ __forceinline__ double fix_per_mu(double mu) {
  return mu != 0.0 ? mcx::scale_pow2(mcx::recip_rn(fabs(mu)), 32) : 0.0;
}

// Per-lane counters for the lane's current problem (flushed with atomics,
// lane by lane or summed over a converged warp first: a problem's counters
// share a cache line).
struct LaneCounts {
  int prob;
  uint32_t src, flights, coll, absn, scat, llo, lhi, capped, exh;
  uint64_t draws, exd, maxd;
  __device__ void clear() {
    src = flights = coll = absn = scat = llo = lhi = capped = exh = 0u;
    draws = exd = maxd = 0ull;
  }
  __device__ void flush(unsigned long long* counts) {
    if (prob < 0) return;
    unsigned long long* c = counts + (size_t)prob * MC_NCOUNT;
    if (src) atomicAdd(c + MC_C_SOURCE, (unsigned long long)src);
    if (flights) atomicAdd(c + MC_C_FLIGHTS, (unsigned long long)flights);
    if (coll) atomicAdd(c + MC_C_COLLISIONS, (unsigned long long)coll);
    if (absn) atomicAdd(c + MC_C_ABSORPTIONS, (unsigned long long)absn);
    if (scat) atomicAdd(c + MC_C_SCATTERS, (unsigned long long)scat);
    if (llo) atomicAdd(c + MC_C_LEAK_LO, (unsigned long long)llo);
    if (lhi) atomicAdd(c + MC_C_LEAK_HI, (unsigned long long)lhi);
    if (draws) atomicAdd(c + MC_C_DRAWS, (unsigned long long)draws);
    if (exh) atomicAdd(c + MC_C_EXCEED_HIST, (unsigned long long)exh);
    if (exd) atomicAdd(c + MC_C_EXCEED_DRAWS, (unsigned long long)exd);
    if (capped) atomicAdd(c + MC_C_CAPPED, (unsigned long long)capped);
    if (maxd) atomicMax(c + MC_C_MAX_DRAWS, (unsigned long long)maxd);
    clear();
  }
  // The same for a whole converged warp: sums first, then one lane's atomics.
  __device__ void flush_warp(unsigned long long* counts) {
    const int p = mcd::warp_common_prob(prob);
    if (p == -2) { flush(counts); return; }
    if (p < 0) return;
    const unsigned long long so = mcd::warp_sum64(src), fl = mcd::warp_sum64(flights), co = mcd::warp_sum64(coll),
                             ab = mcd::warp_sum64(absn), sc = mcd::warp_sum64(scat), lo = mcd::warp_sum64(llo),
                             hi = mcd::warp_sum64(lhi), cp = mcd::warp_sum64(capped), ex = mcd::warp_sum64(exh),
                             dr = mcd::warp_sum64(draws), ed = mcd::warp_sum64(exd), mx = mcd::warp_max64(maxd);
    if ((threadIdx.x & 31u) == 0u) {
      unsigned long long* c = counts + (size_t)p * MC_NCOUNT;
      if (so) atomicAdd(c + MC_C_SOURCE, so);
      if (fl) atomicAdd(c + MC_C_FLIGHTS, fl);
      if (co) atomicAdd(c + MC_C_COLLISIONS, co);
      if (ab) atomicAdd(c + MC_C_ABSORPTIONS, ab);
      if (sc) atomicAdd(c + MC_C_SCATTERS, sc);
      if (lo) atomicAdd(c + MC_C_LEAK_LO, lo);
      if (hi) atomicAdd(c + MC_C_LEAK_HI, hi);
      if (dr) atomicAdd(c + MC_C_DRAWS, dr);
      if (ex) atomicAdd(c + MC_C_EXCEED_HIST, ex);
      if (ed) atomicAdd(c + MC_C_EXCEED_DRAWS, ed);
      if (cp) atomicAdd(c + MC_C_CAPPED, cp);
      if (mx) atomicMax(c + MC_C_MAX_DRAWS, mx);
    }
    clear();
  }
};

// Outcome of a flight or a collision.
enum Outcome : int { kContinue = 0, kAbsorbed = 1, kLeakLo = 2, kLeakHi = 3, kCollide = 4 };

// Source of a history (isotropic uniform in [0, L], or a beam at x = 0).
template <int M, bool F32>
__device__ __forceinline__ void slab_source(const SlabDev& p, Rng<M>& r, const mcd::Lcg& l, SlabParticle& q) {
  if (p.source == MC_SRC_BEAM) {
    q.x = 0.0; q.mu = 1.0; q.w_mu = kFix;
    q.xf = 0.0f; q.xlo = 0.0f; q.muf = 1.0f; q.wf = 1.0f;
    return;
  }
  const double u1 = r.next(l);
  if constexpr (!F32) {
    q.x = __dmul_rn(p.L, u1);
    q.mu = mcx::two_u_minus_1(r.next_n(l));
    q.w_mu = fix_per_mu(q.mu);
  } else {
    // x = L u as the fp64 path has it, split into two floats
    const double x64 = __dmul_rn(p.L, u1);
    q.xf = __double2float_rn(x64);
    q.xlo = __double2float_rn(__dsub_rn(x64, (double)q.xf));
    q.muf = mu_f32(r.next_n(l));
    q.wf = q.muf != 0.0f ? __frcp_rn(fabsf(q.muf)) : 0.0f;
  }
}

// The end of a flight of the fp64 path: xn = x + pm (pm = d mu, rounded
// once), and whether it leaves the slab.  mu is never -0 (2u - 1 rounds an
// exact zero to +0), so its sign is the sign of its bit pattern; x, L and
// the positions of a forward flight are non-negative.
__device__ __forceinline__ int advance64(const SlabDev& p, double x, double mu, double pm, double& xn) {
  xn = __dadd_rn(x, pm);
  const long long mb = __double_as_longlong(mu);
  if (mb > 0 && !nn_lt(xn, p.L)) return kLeakHi;
  if (mb < 0 && __double_as_longlong(xn) <= 0) return kLeakLo;
  return kCollide;
}

// advance64's face tests alone: whether xn, the end of a flight with
// direction bits mb, lies outside the slab.
__device__ __forceinline__ bool leaves64(const SlabDev& p, long long mb, double xn) {
  return (mb > 0 && !nn_lt(xn, p.L)) || (mb < 0 && __double_as_longlong(xn) <= 0);
}

// The tally of that flight: the track from x to xn, to the face it leaves
// through, or (mu = 0) the whole distance d in the bin holding x.  Every
// kind of flight ends in the one call of the bin walk, with its ends chosen
// first, so that the lanes of a warp whose flights differ in kind still walk
// the bins together.
__device__ __forceinline__ void tally64(const SlabDev& p, double x, double xn, double mu, double d, double w_mu,
                                        int outcome, const Sink& s) {
  const long long mb = __double_as_longlong(mu);
  if (outcome == kCollide && mb == 0) { point64(p, x, d, s); return; }
  double a = x, b = xn;                          // forward flight
  if (outcome == kLeakHi) b = p.L;
  else if (outcome == kLeakLo) { a = 0.0; b = x; }
  else if (mb < 0) { a = xn; b = x; }            // backward flight
  seg64(p, a, b, w_mu, s);
}

// The fp32 path's position step: xn + xnlo = (xf + xlo) + d muf, with pr =
// d muf rounded and pe its exact error (a fused multiply-add); the sum by
// TwoSum, the low parts' sum rounded once more (a second-order error).
__device__ __forceinline__ void pair_step(float xf, float xlo, float pr, float pe, float& xn, float& xnlo) {
  float s0, t0;
  two_sum_f(xf, pr, s0, t0);
  two_sum_f(s0, __fadd_rn(t0, __fadd_rn(xlo, pe)), xn, xnlo);
}

// The pair's end point is inside the slab and outside the guard bands: the
// flight collides there (advance32 decides the same, with the same xn, xnlo).
__device__ __forceinline__ bool plain_collision32(const SlabDev& p, float muf, float xn, float xnlo) {
  const bool near_hi = muf > 0.0f && fabsf(xn - p.L_f) <= p.guard_f;
  const bool near_lo = muf < 0.0f && fabsf(xn) <= p.guard_f;
  const bool leak_hi = muf > 0.0f && (xn > p.L_f || (xn == p.L_f && xnlo >= 0.0f));
  const bool leak_lo = muf < 0.0f && (xn < 0.0f || (xn == 0.0f && xnlo <= 0.0f));
  return !(near_hi | near_lo | leak_hi | leak_lo);
}

// The end of a flight of the fp32 path by pair_step, and whether it leaves
// the slab; near a face the leak-or-collide decision is made again in fp64
// from the flight's uniform, uf() (called only there).
template <class UF>
__device__ __forceinline__ int advance32(const SlabDev& p, float xf, float xlo, float muf, float pr, float pe,
                                         UF uf, float& xn, float& xnlo) {
  pair_step(xf, xlo, pr, pe, xn, xnlo);
  // Guard band: re-decide leak vs collide in fp64 near a face.
  const bool near_hi = muf > 0.0f && fabsf(xn - p.L_f) <= p.guard_f;
  const bool near_lo = muf < 0.0f && fabsf(xn) <= p.guard_f;
  // xn + xnlo >= L (or <= 0) from the pair: the low part decides a tie of the high part
  bool leak_hi = muf > 0.0f && (xn > p.L_f || (xn == p.L_f && xnlo >= 0.0f));
  bool leak_lo = muf < 0.0f && (xn < 0.0f || (xn == 0.0f && xnlo <= 0.0f));
  if (near_hi || near_lo) {
    const double d64 = __dmul_rn(-mclog::log1m(uf()), p.inv_st);
    const double x64 = __dadd_rn((double)xf, (double)xlo);
    const double xn64 = __dadd_rn(x64, __dmul_rn(d64, (double)muf));
    leak_hi = muf > 0.0f && xn64 >= p.L;
    leak_lo = muf < 0.0f && xn64 <= 0.0;
    xn = __double2float_rn(xn64);
    if (!leak_hi && !leak_lo) {
      // keep the collision site's high part strictly inside
      if (xn >= p.L_f) xn = __int_as_float(__float_as_int(p.L_f) - 1);
      if (xn <= 0.0f) xn = 1.0e-30f;
    }
    xnlo = __double2float_rn(__dsub_rn(xn64, (double)xn));
  }
  return leak_hi ? kLeakHi : (leak_lo ? kLeakLo : kCollide);
}

// tally64's counterpart for the fp32 path, on position pairs.
__device__ __forceinline__ void tally32(const SlabDev& p, float xf, float xlo, float xn, float xnlo, float muf,
                                        float d, float wf, int outcome, const Sink& s) {
  if (outcome == kCollide && muf == 0.0f) { point32(p, xf, d, s); return; }
  float ah = xf, al = xlo, bh = xn, bl = xnlo;   // forward flight
  if (outcome == kLeakHi) { bh = p.L_f; bl = 0.0f; }
  else if (outcome == kLeakLo) { ah = 0.0f; al = 0.0f; bh = xf; bl = xlo; }
  else if (muf < 0.0f) { ah = xn; al = xnlo; bh = xf; bl = xlo; }  // backward flight
  seg32(p, ah, al, bh, bl, wf, s);
}

// One flight: sample the distance, tally the track, and either leak
// (kLeakLo / kLeakHi) or stop at the collision site (kCollide).
template <int M, bool F32>
__device__ __forceinline__ int slab_flight(const SlabDev& p, Rng<M>& r, const mcd::Lcg& l, SlabParticle& q,
                                           const Sink& s) {
  if constexpr (!F32) {
    const double d = __dmul_rn(-mclog::log1m_n(r.next_n(l)), p.inv_st);
    double xn;
    const int f = advance64(p, q.x, q.mu, __dmul_rn(d, q.mu), xn);
    tally64(p, q.x, xn, q.mu, d, q.w_mu, f, s);
    if (f == kCollide) q.x = xn;
    return f;
  } else {
    const double u = r.next(l);
    const float d = flight_f32(u) * p.inv_st_f;
    const float pr = __fmul_rn(d, q.muf);
    const float pe = __fmaf_rn(d, q.muf, -pr);
    float xn, xnlo;
    const int f = advance32(p, q.xf, q.xlo, q.muf, pr, pe, [u] { return u; }, xn, xnlo);
    tally32(p, q.xf, q.xlo, xn, xnlo, q.muf, d, q.wf, f, s);
    if (f == kCollide) {
      q.xf = xn;
      q.xlo = xnlo;
    }
    return f;
  }
}

// One collision at the current site: absorption (kAbsorbed) or isotropic
// scattering into a new direction (kContinue).
template <int M, bool F32>
__device__ __forceinline__ int slab_collide(const SlabDev& p, Rng<M>& r, const mcd::Lcg& l, SlabParticle& q) {
  if (r.next_n(l) < p.p_abs_n) return kAbsorbed;  // u < 1 - c
  if constexpr (!F32) {
    q.mu = mcx::two_u_minus_1(r.next_n(l));
    q.w_mu = fix_per_mu(q.mu);
  } else {
    q.muf = mu_f32(r.next_n(l));
    q.wf = q.muf != 0.0f ? __frcp_rn(fabsf(q.muf)) : 0.0f;
  }
  return kContinue;
}

// One flight and, if the particle stays in the slab, one collision (the
// history-based step).  Counts collisions and scatters into *coll, *scat.
template <int M, bool F32>
__device__ __forceinline__ int slab_event(const SlabDev& p, Rng<M>& r, const mcd::Lcg& l, SlabParticle& q,
                                          const Sink& s, uint32_t& coll, uint32_t& scat) {
  const int f = slab_flight<M, F32>(p, r, l, q, s);
  if (f != kCollide) return f;
  ++coll;
  const int c = slab_collide<M, F32>(p, r, l, q);
  if (c == kContinue) ++scat;
  return c;
}

}  // namespace mcs

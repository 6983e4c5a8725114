// box.cuh -- device physics of the two-region multigroup box, shared by the
// history-based (box.cu) and event-based (box_event.cu) schedules.
//
// Geometry: box [0,S]^3 with an inner cube [lo,hi]^3 (region 1) inside the
// outer region 0, vacuum outside.  Surface tracking: each flight samples
// d = -ln(1-u) / Sigma_t[region] and stops at the region surface if that is
// nearer.  Collisions: implicit capture, downscatter by CDF row, isotropic
// direction by Marsaglia's rejection method, then the region's weight window
// (roulette or split).  Children of a split are seeded on demand with
// S_c = hash(k, S_p) (Section 4, Eq. 5) from the parent's current state.
// Track lengths go to a group-summed mesh as int64 fixed point (2^32).
//
// T = double: every operation rounds once (this code is compiled with
// --fmad=false), matching the fp64 transport definition step for step.
// T = float: geometry and distances in fp32; a flight whose fp32 collision
// distance lies within a relative 2^-16 of the surface distance is decided
// again in fp64; uniforms, hashes and the fixed-point scaling stay exact.
#pragma once
#include <cstdint>

#include "../../include/mc.h"
#include "mc_device.cuh"
#include "slab.cuh"

namespace mcb {

constexpr int kMaxG = MC_BOX_MAX_GROUPS;

struct BoxDev {
  double side, lo, hi;
  double st[2], c[2], wl[2], wh[2], ws[2];
  double cdf[2][kMaxG][kMaxG];
  uint64_t n_hist, seed, stride_q, id_offset, key, tally_offset;
  uint32_t ng, mesh, max_split, n_batches, seeding, source;
  // derived on the device (box_prep_kernel)
  double inv_st[2], h, inv_h;
  uint32_t ih_q;  // inv_h as ih_q 2^-ih_s: the voxel lookup guess
  int ih_s;
  float side_f, lo_f, hi_f, h_f, inv_h_f;
  float inv_st_f[2], c_f[2], wl_f[2], wh_f[2], ws_f[2];
  uint64_t seed_hash, hist_begin;
};

// A particle of the box (position, direction and its componentwise inverse,
// weight, group, region).
template <typename T>
struct Part {
  T p[3], u[3], inv[3];
  T w;
  uint32_t g, region;
};

// Record of a split child waiting in a device bank (fp64 fields; fp32
// particles store their values exactly).
struct ChildRec {
  double p[3], u[3], w;
  uint64_t rng;
  uint64_t tbase;  // tally slot row of the family (problem offset + batch row)
  uint32_t g, region, prob, pad;
};

enum BoxOutcome : int { kBoxCollide = 0, kBoxCross = 1, kBoxLeak = 2, kBoxContinue = 3, kBoxKilled = 4 };

template <typename T> __device__ __forceinline__ T from_u(double u);
template <> __device__ __forceinline__ double from_u<double>(double u) { return u; }
template <> __device__ __forceinline__ float from_u<float>(double u) { return (float)u; }

template <typename T> __device__ __forceinline__ T sel(const double& d, const float& f);
template <> __device__ __forceinline__ double sel<double>(const double& d, const float&) { return d; }
template <> __device__ __forceinline__ float sel<float>(const double&, const float& f) { return f; }

// Comparisons: fp64 on the integer pipes (sign-magnitude order keys, equal to
// the fp64 comparisons for non-NaN values), fp32 native.
__device__ __forceinline__ bool lt(double a, double b) { return mcx::d_lt(a, b); }
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ bool eq(double a, double b) { return mcx::okey(a) == mcx::okey(b); }
__device__ __forceinline__ bool eq(float a, float b) { return a == b; }
__device__ __forceinline__ bool gt0(double a) { return mcx::d_pos(a); }
__device__ __forceinline__ bool gt0(float a) { return a > 0.0f; }
__device__ __forceinline__ bool lt0(double a) { return mcx::d_neg(a); }
__device__ __forceinline__ bool lt0(float a) { return a < 0.0f; }
__device__ __forceinline__ bool is0(double a) { return mcx::d_zero(a); }
__device__ __forceinline__ bool is0(float a) { return a == 0.0f; }

template <typename T> __device__ __forceinline__ T recip(T v);
template <> __device__ __forceinline__ double recip<double>(double v) { return mcx::recip_rn(v); }
template <> __device__ __forceinline__ float recip<float>(float v) { return 1.0f / v; }

// Componentwise inverse of the direction (fp64: the correctly rounded
// reciprocal on the integer pipes, fp_exact.cuh).
template <typename T>
__device__ __forceinline__ void set_inv(Part<T>& q) {
#pragma unroll 1
  for (int a = 0; a < 3; ++a) q.inv[a] = !is0(q.u[a]) ? recip<T>(q.u[a]) : T(0);
}

// Marsaglia (1972): v1, v2 uniform on [-1,1)^2 until v1^2 + v2^2 < 1.
template <int M, typename T>
__device__ __forceinline__ void iso_dir(mcs::Rng<M>& r, const mcd::Lcg& l, T u[3]) {
  T v1, v2, s;
  do {
    if constexpr (sizeof(T) == 8) {  // 2u - 1 exactly, on the integer pipes
      v1 = mcx::two_u_minus_1(r.next_n(l));
      v2 = mcx::two_u_minus_1(r.next_n(l));
    } else {
      v1 = T(2) * from_u<T>(r.next(l)) - T(1);
      v2 = T(2) * from_u<T>(r.next(l)) - T(1);
    }
    s = v1 * v1 + v2 * v2;
  } while (!lt(s, T(1)));
  const T t = sqrt(T(1) - s);
  u[0] = T(2) * v1 * t;
  u[1] = T(2) * v2 * t;
  u[2] = T(1) - T(2) * s;
}

template <typename T>
__device__ __forceinline__ uint32_t region_of(const BoxDev& b, const T p[3], const T u[3]) {
  const T lo = sel<T>(b.lo, b.lo_f), hi = sel<T>(b.hi, b.hi_f);
  for (int a = 0; a < 3; ++a) {
    const bool above = lt(lo, p[a]) || (eq(p[a], lo) && gt0(u[a]));
    const bool below = lt(p[a], hi) || (eq(p[a], hi) && lt0(u[a]));
    if (!above || !below) return 0u;
  }
  return 1u;
}

template <typename T>
__device__ __forceinline__ T exit_dist(const Part<T>& q, T lo, T hi) {
  T t = T(INFINITY);
  for (int a = 0; a < 3; ++a) {
    T ta;
    if (gt0(q.u[a])) ta = (hi - q.p[a]) * q.inv[a];
    else if (lt0(q.u[a])) ta = (lo - q.p[a]) * q.inv[a];
    else continue;
    if (lt(ta, t)) t = ta;
  }
  return lt0(t) ? T(0) : t;
}

template <typename T>
__device__ __forceinline__ T entry_dist(const Part<T>& q, T lo, T hi) {
  T tn = T(-INFINITY), tf = T(INFINITY);
  for (int a = 0; a < 3; ++a) {
    if (!is0(q.u[a])) {
      const T t1 = (lo - q.p[a]) * q.inv[a], t2 = (hi - q.p[a]) * q.inv[a];
      const bool o = lt(t1, t2);
      const T tmin = o ? t1 : t2, tmax = o ? t2 : t1;
      if (lt(tn, tmin)) tn = tmin;
      if (lt(tmax, tf)) tf = tmax;
    } else if (!lt(lo, q.p[a]) || !lt(q.p[a], hi)) {
      return T(INFINITY);
    }
  }
  if (!lt0(tn) && lt(tn, tf)) return tn;
  return T(INFINITY);
}

// Distance to the region surface and its kind (1: into the other region,
// 2: out of the box).
template <typename T>
__device__ __forceinline__ T surface(const BoxDev& b, const Part<T>& q, int& kind) {
  const T lo = sel<T>(b.lo, b.lo_f), hi = sel<T>(b.hi, b.hi_f), side = sel<T>(b.side, b.side_f);
  if (q.region == 1u) {
    kind = 1;
    return exit_dist(q, lo, hi);
  }
  const T de = entry_dist(q, lo, hi);
  const T dx = exit_dist(q, T(0), side);
  const bool in = lt(de, dx);
  kind = in ? 1 : 2;
  return in ? de : dx;
}

__device__ __forceinline__ long long fix_of(double wl) { return mcx::fix32_nonneg(wl); }
__device__ __forceinline__ long long fix_of(float wl) { return mcs::fix32_from_float(wl); }

// Mesh plane j: RN(j h) for j < mesh, side for j = mesh.  fp64: from the
// caller's table (shared memory, one problem per launch) or computed as one
// rounding of an exact integer product (mesh <= 1024).
constexpr int kMaxPlanes = MC_BOX_MAX_MESH + 1;
__device__ __forceinline__ double plane_of(const BoxDev& b, int j) {
  return j >= (int)b.mesh ? b.side : mcx::mul_small((uint32_t)j, b.h);
}
template <typename T> __device__ __forceinline__ T plane(const BoxDev& b, const double* tab, int j);
template <> __device__ __forceinline__ double plane<double>(const BoxDev& b, const double* tab, int j) {
  return tab ? tab[j] : plane_of(b, j);
}
template <> __device__ __forceinline__ float plane<float>(const BoxDev& b, const double*, int j) {
  return j >= (int)b.mesh ? b.side_f : (float)j * b.h_f;
}

template <typename T> __device__ __forceinline__ int voxel_guess(const BoxDev& b, T p);
template <> __device__ __forceinline__ int voxel_guess<double>(const BoxDev& b, double p) {
  return lt0(p) ? -1 : (int)min(mcx::guess_floor_mul(p, b.ih_q, b.ih_s), (uint64_t)b.mesh);
}
template <> __device__ __forceinline__ int voxel_guess<float>(const BoxDev& b, float p) {
  return (int)floorf(p * b.inv_h_f);
}

// Track-length tally of p + t u, 0 <= t <= L, by a voxel walk: the next
// crossing on each axis is computed from the segment start directly,
// t = (plane - p) / u, so every piece has the length the clipping definition
// gives it.  base: this history's [mesh^3] slot row.
template <typename T>
__device__ void trace(const BoxDev& b, const Part<T>& q, T L, unsigned long long* base, const double* tab,
                      bool agg) {
  const int nm = (int)b.mesh;
  const T h = sel<T>(b.h, b.h_f), inv_h = sel<T>(b.inv_h, b.inv_h_f);
  int idx[3];
  T tn[3];
  for (int a = 0; a < 3; ++a) {
    int i = voxel_guess<T>(b, q.p[a]);
    i = i < 0 ? 0 : (i >= nm ? nm - 1 : i);
    while (i > 0 && lt(q.p[a], plane<T>(b, tab, i))) --i;
    while (i + 1 < nm && !lt(q.p[a], plane<T>(b, tab, i + 1))) ++i;
    if (lt0(q.u[a]) && i > 0 && eq(q.p[a], plane<T>(b, tab, i))) --i;
    idx[a] = i;
    if (gt0(q.u[a])) tn[a] = (plane<T>(b, tab, i + 1) - q.p[a]) * q.inv[a];
    else if (lt0(q.u[a])) tn[a] = (plane<T>(b, tab, i) - q.p[a]) * q.inv[a];
    else tn[a] = T(INFINITY);
  }
  (void)h;
  (void)inv_h;
  T t = T(0);
  const T w = q.w;
  for (int guard = 0; guard < 3 * nm + 8; ++guard) {
    int a = 0;
    if (lt(tn[1], tn[a])) a = 1;
    if (lt(tn[2], tn[a])) a = 2;
    const bool inside = lt(tn[a], L);
    const T tend = inside ? tn[a] : L;
    if (lt(t, tend)) {
      const long long v = fix_of(w * (tend - t));
      if (v != 0) {
        const uint64_t slot = ((uint64_t)idx[2] * nm + idx[1]) * nm + idx[0];
        if (agg) mcd::warp_agg_add(base + slot, (unsigned long long)v);
        else atomicAdd(base + slot, (unsigned long long)v);
      }
      t = tend;
    }
    if (!inside) break;
    // step across the plane on axis a
    if (gt0(q.u[a])) {
      idx[a] += 1;
      if (idx[a] >= nm) break;
      tn[a] = (plane<T>(b, tab, idx[a] + 1) - q.p[a]) * q.inv[a];
    } else {
      idx[a] -= 1;
      if (idx[a] < 0) break;
      tn[a] = (plane<T>(b, tab, idx[a]) - q.p[a]) * q.inv[a];
    }
  }
}

template <int M, typename T>
__device__ __forceinline__ void box_source(const BoxDev& b, mcs::Rng<M>& r, const mcd::Lcg& l, Part<T>& q) {
  const T side = sel<T>(b.side, b.side_f);
  for (int a = 0; a < 3; ++a) q.p[a] = side * from_u<T>(r.next(l));
  iso_dir<M, T>(r, l, q.u);
  set_inv(q);
  q.w = T(1);
  q.g = 0u;
  q.region = region_of<T>(b, q.p, q.u);
}

// One flight: collide (position moved to the site), cross into the other
// region (moved to the surface), or leak out of the box.
template <int M, typename T>
__device__ __forceinline__ int box_flight(const BoxDev& b, mcs::Rng<M>& r, const mcd::Lcg& l, Part<T>& q,
                                          unsigned long long* base, const double* tab, bool agg) {
  int kind = 0;
  T ds = surface<T>(b, q, kind);
  bool collide;
  T d;
  if constexpr (sizeof(T) == 8) {
    d = -mclog::log1m_n(r.next_n(l)) * b.inv_st[q.region];
    collide = lt(d, ds);
  } else {
    const double u = r.next(l);
    d = mcs::flight_f32(u) * b.inv_st_f[q.region];
    collide = d < ds;
    if (fabsf(d - ds) <= 0x1p-16f * fmaxf(d, ds)) {  // near the surface: decide in fp64
      Part<double> q64;
      for (int a = 0; a < 3; ++a) {
        q64.p[a] = q.p[a];
        q64.u[a] = q.u[a];
        q64.inv[a] = q.inv[a] != 0.0f ? mcx::recip_rn((double)q.u[a]) : 0.0;
      }
      q64.region = q.region;
      int k64 = 0;
      const double ds64 = surface<double>(b, q64, k64);
      const double d64 = -mclog::log1m(u) * b.inv_st[q.region];
      collide = d64 < ds64;
      kind = k64;
    }
  }
  const T len = collide ? d : ds;
  trace<T>(b, q, len, base, tab, agg);
  for (int a = 0; a < 3; ++a) q.p[a] = q.p[a] + len * q.u[a];
  if (collide) return kBoxCollide;
  if (kind == 2) return kBoxLeak;
  q.region ^= 1u;
  return kBoxCross;
}

// One collision: implicit capture, group, direction, weight window.
// Returns kBoxContinue, kBoxKilled (roulette), or the number n >= 2 of
// particles of a split (the parent keeps weight w/n; the caller creates the
// n-1 children from the parent's state after this call).
template <int M, typename T>
__device__ __forceinline__ int box_collide(const BoxDev& b, mcs::Rng<M>& r, const mcd::Lcg& l, Part<T>& q) {
  const uint32_t rg = q.region;
  q.w = q.w * sel<T>(b.c[rg], b.c_f[rg]);
  const double ug = r.next(l);
  uint32_t g2 = q.g;
  for (uint32_t k = q.g; k < b.ng; ++k) {
    if (mcs::nn_lt(ug, b.cdf[rg][q.g][k])) {  // both non-negative
      g2 = k;
      break;
    }
  }
  q.g = g2;
  iso_dir<M, T>(r, l, q.u);
  set_inv(q);
  const T wl = sel<T>(b.wl[rg], b.wl_f[rg]), wh = sel<T>(b.wh[rg], b.wh_f[rg]);
  if (lt(q.w, wl)) {
    const T ws = sel<T>(b.ws[rg], b.ws_f[rg]);
    if (lt(from_u<T>(r.next(l)), q.w / ws)) {
      q.w = ws;
      return kBoxContinue;
    }
    return kBoxKilled;
  }
  if (lt(wh, q.w)) {
    const T nd = ceil(q.w / wh);
    const uint32_t ns = nd > (T)b.max_split ? b.max_split : (uint32_t)nd;
    if (ns > 1u) {
      q.w = q.w / (T)ns;
      return (int)ns + 8;  // encoded: n + 8 (> every other outcome)
    }
  }
  return kBoxContinue;
}

// Per-lane counters of one problem, flushed with atomics (lane by lane, or
// summed over a converged warp first: a problem's counters share a cache line).
struct BoxCounts {
  int prob;
  uint32_t src, flights, coll, leaks, kills, splits, children, capped, exh;
  uint64_t draws, exd, maxd;
  __device__ void clear() {
    src = flights = coll = leaks = kills = splits = children = capped = exh = 0u;
    draws = exd = maxd = 0ull;
  }
  __device__ void flush(unsigned long long* counts) {
    if (prob < 0) return;
    unsigned long long* c = counts + (size_t)prob * MC_NCOUNT;
    if (src) atomicAdd(c + MC_C_SOURCE, (unsigned long long)src);
    if (flights) atomicAdd(c + MC_C_FLIGHTS, (unsigned long long)flights);
    if (coll) {
      atomicAdd(c + MC_C_COLLISIONS, (unsigned long long)coll);
      atomicAdd(c + MC_C_SCATTERS, (unsigned long long)coll);
    }
    if (leaks) atomicAdd(c + MC_C_LEAK_HI, (unsigned long long)leaks);
    if (kills) atomicAdd(c + MC_C_ROULETTE_KILLS, (unsigned long long)kills);
    if (splits) atomicAdd(c + MC_C_SPLITS, (unsigned long long)splits);
    if (children) atomicAdd(c + MC_C_CHILDREN, (unsigned long long)children);
    if (capped) atomicAdd(c + MC_C_CAPPED, (unsigned long long)capped);
    if (exh) atomicAdd(c + MC_C_EXCEED_HIST, (unsigned long long)exh);
    if (draws) atomicAdd(c + MC_C_DRAWS, (unsigned long long)draws);
    if (exd) atomicAdd(c + MC_C_EXCEED_DRAWS, (unsigned long long)exd);
    if (maxd) atomicMax(c + MC_C_MAX_DRAWS, (unsigned long long)maxd);
    clear();
  }
  // The same for a whole converged warp: sums first, then one lane's atomics
  // (a problem's counters share a cache line).
  __device__ void flush_warp(unsigned long long* counts) {
    const int p = mcd::warp_common_prob(prob);
    if (p == -2) { flush(counts); return; }
    if (p < 0) return;
    const unsigned long long so = mcd::warp_sum64(src), fl = mcd::warp_sum64(flights), co = mcd::warp_sum64(coll),
                             le = mcd::warp_sum64(leaks), ki = mcd::warp_sum64(kills), sp = mcd::warp_sum64(splits),
                             ch = mcd::warp_sum64(children), cp = mcd::warp_sum64(capped), ex = mcd::warp_sum64(exh),
                             dr = mcd::warp_sum64(draws), ed = mcd::warp_sum64(exd), mx = mcd::warp_max64(maxd);
    if ((threadIdx.x & 31u) == 0u) {
      unsigned long long* c = counts + (size_t)p * MC_NCOUNT;
      if (so) atomicAdd(c + MC_C_SOURCE, so);
      if (fl) atomicAdd(c + MC_C_FLIGHTS, fl);
      if (co) {
        atomicAdd(c + MC_C_COLLISIONS, co);
        atomicAdd(c + MC_C_SCATTERS, co);
      }
      if (le) atomicAdd(c + MC_C_LEAK_HI, le);
      if (ki) atomicAdd(c + MC_C_ROULETTE_KILLS, ki);
      if (sp) atomicAdd(c + MC_C_SPLITS, sp);
      if (ch) atomicAdd(c + MC_C_CHILDREN, ch);
      if (cp) atomicAdd(c + MC_C_CAPPED, cp);
      if (ex) atomicAdd(c + MC_C_EXCEED_HIST, ex);
      if (dr) atomicAdd(c + MC_C_DRAWS, dr);
      if (ed) atomicAdd(c + MC_C_EXCEED_DRAWS, ed);
      if (mx) atomicMax(c + MC_C_MAX_DRAWS, mx);
    }
    clear();
  }
};

constexpr int kSplitBase = 8;

// Child k of a split: Eq. (5), S_c = hash(k, S_p) mod 2^m.
__device__ __forceinline__ uint64_t child_seed(uint32_t k, uint64_t parent_state, uint64_t mask) {
  return mcd::hash64((uint64_t)k, parent_state & mask) & mask;
}

template <typename T>
__device__ __forceinline__ void store_child(ChildRec& c, const Part<T>& q, uint64_t seed, uint32_t prob,
                                            uint64_t tbase) {
  for (int a = 0; a < 3; ++a) {
    c.p[a] = (double)q.p[a];
    c.u[a] = (double)q.u[a];
  }
  c.w = (double)q.w;
  c.rng = seed;
  c.tbase = tbase;
  c.g = q.g;
  c.region = q.region;
  c.prob = prob;
  c.pad = 0;
}

template <typename T>
__device__ __forceinline__ void load_child(const ChildRec& c, Part<T>& q) {
  for (int a = 0; a < 3; ++a) {
    q.p[a] = (T)c.p[a];
    q.u[a] = (T)c.u[a];
  }
  q.w = (T)c.w;
  q.g = c.g;
  q.region = c.region;
  set_inv(q);
}

}  // namespace mcb

// pulse.cuh -- device record and seeds of the pulse problem (Section 5),
// shared by the single-run kernel (pulse.cu) and the census-phase kernel
// (pulse_census.cu).
#pragma once
#include <cstdint>

#include "../../include/mc.h"
#include "mc_device.cuh"
#include "slab.cuh"

namespace mcp {

struct PulseDev {
  double c, nu, t_end, x_half, sigma_t;
  uint64_t n_hist, seed, stride_q, id_offset, tally_offset;
  uint32_t n_reps, n_batches, per_batch, n_time_bins, seeding, n_census, pc_target, pad;
  // derived by pulse_prep_kernel
  double inv_st;
  long long unit;      // llrint(2^32 / Sigma_t): one collision-estimator score
  uint64_t seed_hash;  // flat hash mode: seed half of hash(., s)
  // the draws' tests as integer thresholds on n (u = n 2^-53):
  uint64_t c_n;        // u < c            <=>  n < c_n = ceil(c 2^53)
  uint64_t nu_n;       // floor(nu + u) = nu_floor + (n >= nu_n)
  uint32_t nu_floor, pad2;
};

constexpr int kStack = 256;  // most pending secondaries a lane keeps (run config stack_depth)

// A pending secondary on a lane's local stack (census phases: shallow
// families, where the L1-resident local stack measured faster).
struct Pending {
  double x, t;
  uint64_t seed;
};

// A pending secondary in device memory (one 32-byte sector): the stacks of
// all lanes of a launch, depth-major (entry j of every lane together), so a
// push writes one whole sector and the shallow entries, the busy ones, stay
// together in L2.
struct __align__(32) StackRec {
  double x, t;
  uint64_t seed, pad;
};
__device__ __forceinline__ void stack_put(StackRec* e, double x, double t, uint64_t seed) {
  reinterpret_cast<double2*>(e)[0] = make_double2(x, t);
  reinterpret_cast<ulonglong2*>(e)[1] = make_ulonglong2(seed, 0ull);
}
__device__ __forceinline__ void stack_get(const StackRec* e, double& x, double& t, uint64_t& seed) {
  const double2 v = reinterpret_cast<const double2*>(e)[0];
  x = v.x;
  t = v.y;
  seed = reinterpret_cast<const ulonglong2*>(e)[1].x;
}

// A hash-seeded secondary that did not fit on its lane's stack (32 bytes):
// it waits in a device bank for a later launch of the same phase.
struct Overflow {
  double x, t;
  uint64_t seed;
  uint32_t group;  // rep * n_batches + batch: its tally row
  uint32_t pad;
};

__device__ __forceinline__ uint64_t pulse_seed(const PulseDev& P, uint64_t g, const mcd::Affine* tab,
                                               uint64_t mask) {
  if (P.seeding == MC_SEED_STRIDE) return mcs::skip_tab(tab, P.seed, P.stride_q * (P.id_offset + g)) & mask;
  if (P.seeding == MC_SEED_HASH) return mcd::hash_with(g, P.seed_hash) & mask;
  const uint64_t pb = P.per_batch, nb = P.n_batches;
  const uint64_t rep = g / (pb * nb), batch = (g / pb) % nb, part = g % pb;
  const uint64_t h_rep = mcd::hash64(rep, P.seed);
  return mcd::hash64(part, mcd::hash64(batch, h_rep)) & mask;
}

}  // namespace mcp

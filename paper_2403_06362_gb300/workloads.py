"""Seeded synthetic workloads: problem parameters only, no method arithmetic.

This module is the one place both the CUDA path and the CPU oracle take
their inputs from.  It holds plain parameter records (dicts) and draws the
random problem parameters of the batched workload with numpy's seeded
generator; it never evaluates an LCG step, a hash, a skip-ahead or any
transport physics.

Workloads (all synthetic, shapes of the paper's setting, Sections 3-5):
  slab_small      1D slab L = 10 cm, Sigma_t = 1/cm, c = 0.5, isotropic source
                  uniform in [0, L], vacuum, 10^4 histories, 20 bins, 10 batches
  rng_microbench  2^26 streams (history ids 0..2^26-1), seed 42 / X0 = 1,
                  Q = 152917, 64 uniforms per stream
  slab_batched    256 slab problems from numpy seed 7: histories log-uniform in
                  [10^3, 10^6], L ~ U[1, 50] cm, Sigma_t ~ U[0.5, 2]/cm,
                  c ~ U[0.1, 0.99], 64 bins each, hierarchical hash seeds
                  hash(j, hash(i, 42)) or stride with global unit ids
  slab_long       1D slab L = 200 cm, Sigma_t = 1/cm, c = 0.9999, 10^6 histories,
                  200 bins, 20 batches
"""
from __future__ import annotations

import numpy as np

LCG_M, LCG_G, LCG_C = 63, 2806196910506780709, 1
STRIDE_Q = 152917
HASH_SEED = 42
STRIDE_X0 = 1

SEED_HASH, SEED_STRIDE, SEED_HASH_HIER = 0, 1, 2
SRC_ISOTROPIC, SRC_BEAM = 0, 1


def slab_problem(L, sigma_t, c, n_histories, n_bins, n_batches, seeding, source=SRC_ISOTROPIC,
                 tally_offset=0, id_offset=0, key=0, seed=None, stride_q=STRIDE_Q):
    if seed is None:
        seed = STRIDE_X0 if seeding == SEED_STRIDE else HASH_SEED
    return dict(L=float(L), sigma_t=float(sigma_t), c=float(c), n_histories=int(n_histories),
                n_bins=int(n_bins), n_batches=int(n_batches), seeding=int(seeding),
                source=int(source), tally_offset=int(tally_offset), id_offset=int(id_offset),
                key=int(key), seed=int(seed), stride_q=int(stride_q))


def tally_slots(problems):
    return max(p["tally_offset"] + p["n_bins"] * p["n_batches"] for p in problems)


def slab_small(seeding=SEED_HASH, n_histories=10**4):
    return [slab_problem(10.0, 1.0, 0.5, n_histories, 20, 10, seeding)]


def slab_long(seeding=SEED_HASH, n_histories=10**6):
    return [slab_problem(200.0, 1.0, 0.9999, n_histories, 200, 20, seeding)]


def slab_batched(seeding=SEED_HASH_HIER, n_problems=256, seed=7, n_bins=64, n_batches=1,
                 max_histories=None):
    """256 uneven slab problems drawn from numpy's generator with `seed`."""
    rng = np.random.default_rng(seed)
    u = rng.random((n_problems, 4))
    probs = []
    off = 0
    ids = 0
    for i in range(n_problems):
        nh = int(np.floor(10.0 ** (3.0 + 3.0 * u[i, 0])))
        if max_histories is not None:
            nh = min(nh, max_histories)
        p = slab_problem(1.0 + 49.0 * u[i, 1], 0.5 + 1.5 * u[i, 2], 0.1 + 0.89 * u[i, 3], nh,
                         n_bins, n_batches, seeding, tally_offset=off,
                         id_offset=ids if seeding == SEED_STRIDE else 0, key=i)
        probs.append(p)
        off += n_bins * n_batches
        ids += nh
    return probs


def rng_microbench(n_streams=2**26, draws=64):
    return dict(n_streams=int(n_streams), draws=int(draws), hash_seed=HASH_SEED,
                stride_x0=STRIDE_X0, stride_q=STRIDE_Q)


def to_mc_problem(p, mc):
    """dict -> libmc's mc_problem (module passed in to keep this file free of imports)."""
    return mc.mc_problem(geometry=mc.MC_GEOM_SLAB, source=p["source"], seeding=p["seeding"],
                         n_bins=p["n_bins"], n_batches=p["n_batches"], reserved=0, L=p["L"],
                         sigma_t=p["sigma_t"], c=p["c"], n_histories=p["n_histories"],
                         seed=p["seed"], stride_q=p["stride_q"], id_offset=p["id_offset"],
                         key=p["key"], tally_offset=p["tally_offset"], box=None)


def to_oracle_problem(p, oracle):
    """dict -> the oracle's SlabProblem (module passed in)."""
    return oracle.SlabProblem(L=p["L"], sigma_t=p["sigma_t"], c=p["c"], n_histories=p["n_histories"],
                              seed=p["seed"], stride_q=p["stride_q"], id_offset=p["id_offset"],
                              key=p["key"], tally_offset=p["tally_offset"], n_bins=p["n_bins"],
                              n_batches=p["n_batches"], source=p["source"], seeding=p["seeding"])


# --- two-region multigroup box ------------------------------------------------
#   box_large  100 cm cube, inner cube [30, 70]^3 (Sigma_t 2.0/cm, c 0.3) in an
#              outer region (Sigma_t 0.5/cm, c 0.95); 4 groups with a
#              downscatter matrix drawn from numpy seed 3; implicit capture;
#              weight windows (w_low, w_high, w_survive): outer (0.25, 2.0, 0.5),
#              inner (0.02, 0.1, 0.05); splits of at most 8; isotropic source
#              uniform in the box, group 0; 64^3 group-summed track-length mesh;
#              10^8 histories, one batch

BOX_MAX_GROUPS = 8


def downscatter_cdf(n_groups=4, seed=3):
    """CDF rows [region][g][g'] of a lower-triangular downscatter matrix
    (g -> g' >= g) with random positive entries; the last group scatters to
    itself only.  Entries below the diagonal are 0; every row ends at 1.0."""
    rng = np.random.default_rng(seed)
    cdf = np.zeros((2, BOX_MAX_GROUPS, BOX_MAX_GROUPS))
    for r in range(2):
        for g in range(n_groups):
            w = rng.random(n_groups - g) + 0.05
            c = np.cumsum(w / w.sum())
            c[-1] = 1.0
            cdf[r, g, g:n_groups] = c
            cdf[r, g, n_groups:] = 1.0
    return cdf


def box_problem(n_histories=10**8, seeding=SEED_HASH, side=100.0, inner=(30.0, 70.0),
                sigma_t=(0.5, 2.0), c=(0.95, 0.3), ww_low=(0.25, 0.02), ww_high=(2.0, 0.1),
                ww_survive=(0.5, 0.05), n_groups=4, mesh=64, max_split=8, n_batches=1,
                tally_offset=0, seed=None, cdf_seed=3):
    if seed is None:
        seed = STRIDE_X0 if seeding == SEED_STRIDE else HASH_SEED
    return dict(side=float(side), inner_lo=float(inner[0]), inner_hi=float(inner[1]),
                sigma_t=tuple(float(v) for v in sigma_t), c=tuple(float(v) for v in c),
                ww_low=tuple(float(v) for v in ww_low), ww_high=tuple(float(v) for v in ww_high),
                ww_survive=tuple(float(v) for v in ww_survive),
                cdf=downscatter_cdf(n_groups, cdf_seed), n_groups=int(n_groups), mesh=int(mesh),
                max_split=int(max_split), n_batches=int(n_batches), n_histories=int(n_histories),
                seeding=int(seeding), seed=int(seed), stride_q=STRIDE_Q, id_offset=0, key=0,
                tally_offset=int(tally_offset), source=SRC_ISOTROPIC)


def box_large(seeding=SEED_HASH, n_histories=10**8):
    return box_problem(n_histories=n_histories, seeding=seeding)


def box_tally_slots(b):
    return b["tally_offset"] + b["n_batches"] * b["mesh"] ** 3


def to_oracle_box(b, oracle):
    o = oracle.BoxProblem()
    o.side, o.inner_lo, o.inner_hi = b["side"], b["inner_lo"], b["inner_hi"]
    for r in range(2):
        o.sigma_t[r], o.c[r] = b["sigma_t"][r], b["c"][r]
        o.ww_low[r], o.ww_high[r], o.ww_survive[r] = b["ww_low"][r], b["ww_high"][r], b["ww_survive"][r]
        for g in range(BOX_MAX_GROUPS):
            for h in range(BOX_MAX_GROUPS):
                o.cdf[r][g][h] = b["cdf"][r, g, h]
    o.n_histories, o.seed, o.stride_q = b["n_histories"], b["seed"], b["stride_q"]
    o.id_offset, o.key, o.tally_offset = b["id_offset"], b["key"], b["tally_offset"]
    o.n_groups, o.mesh, o.max_split, o.n_batches = b["n_groups"], b["mesh"], b["max_split"], b["n_batches"]
    o.seeding, o.source = b["seeding"], b["source"]
    return o


def to_mc_box(b, mc):
    """dict -> (libmc mc_problem, mc_box_spec); keep the spec alive while the
    problem is in use (the problem points to it)."""
    spec = mc.mc_box_spec()
    spec.side, spec.inner_lo, spec.inner_hi = b["side"], b["inner_lo"], b["inner_hi"]
    for r in range(2):
        spec.sigma_t[r], spec.c[r] = b["sigma_t"][r], b["c"][r]
        spec.ww_low[r], spec.ww_high[r], spec.ww_survive[r] = b["ww_low"][r], b["ww_high"][r], b["ww_survive"][r]
        for g in range(BOX_MAX_GROUPS):
            for h in range(BOX_MAX_GROUPS):
                spec.scatter_cdf[r][g][h] = b["cdf"][r, g, h]
    spec.n_groups, spec.mesh, spec.max_split, spec.reserved = b["n_groups"], b["mesh"], b["max_split"], 0
    import ctypes
    prob = mc.mc_problem(geometry=mc.MC_GEOM_BOX, source=b["source"], seeding=b["seeding"],
                         n_bins=b["mesh"] ** 3, n_batches=b["n_batches"], reserved=0, L=b["side"],
                         sigma_t=b["sigma_t"][0], c=b["c"][0], n_histories=b["n_histories"], seed=b["seed"],
                         stride_q=b["stride_q"], id_offset=b["id_offset"], key=b["key"],
                         tally_offset=b["tally_offset"], box=ctypes.pointer(spec))
    return prob, spec


# --- the paper's Section 5 problem (AZURV1-like, supercritical) -----------------
#   azurv1  infinite homogeneous medium, Sigma_t = 1, speed 1, pulse at
#           t = x = 0, scattering ratio 0.4 with multiplicity 2.75 (k = 1.1),
#           census at t = 20; collision-estimator flux averaged over
#           x in [-1, 1] in 20 unit time bins; 30 repetitions x 1000 batches x
#           1000 source particles

def azurv1(seeding=SEED_HASH_HIER, n_reps=30, n_batches=1000, per_batch=1000, c=0.4, nu=2.75, t_end=20.0,
           x_half=1.0, n_time_bins=20, tally_offset=0, seed=None, n_census=0, pc_target=0):
    if seed is None:
        seed = STRIDE_X0 if seeding == SEED_STRIDE else HASH_SEED
    return dict(c=float(c), nu=float(nu), t_end=float(t_end), x_half=float(x_half), sigma_t=1.0,
                seed=int(seed), stride_q=STRIDE_Q, id_offset=0, tally_offset=int(tally_offset),
                n_reps=int(n_reps), n_batches=int(n_batches), per_batch=int(per_batch),
                n_time_bins=int(n_time_bins), seeding=int(seeding), n_census=int(n_census),
                pc_target=int(pc_target))


def azurv1_histories(a):
    return a["n_reps"] * a["n_batches"] * a["per_batch"]


def azurv1_tally_slots(a):
    return a["tally_offset"] + a["n_reps"] * a["n_batches"] * a["n_time_bins"]


def to_oracle_azurv1(a, oracle):
    return oracle.Azurv1Problem(c=a["c"], nu=a["nu"], t_end=a["t_end"], x_half=a["x_half"],
                                sigma_t=a["sigma_t"], seed=a["seed"], stride_q=a["stride_q"],
                                id_offset=a["id_offset"], tally_offset=a["tally_offset"],
                                n_reps=a["n_reps"], n_batches=a["n_batches"], per_batch=a["per_batch"],
                                n_time_bins=a["n_time_bins"], seeding=a["seeding"],
                                n_census=a.get("n_census", 0), pc_target=a.get("pc_target", 0), pad=0)


def to_mc_pulse(a, mc):
    """dict -> (libmc mc_problem, mc_pulse_spec); keep the spec alive while
    the problem is in use."""
    import ctypes
    spec = mc.mc_pulse_spec(c=a["c"], nu=a["nu"], t_end=a["t_end"], x_half=a["x_half"], sigma_t=a["sigma_t"],
                            n_reps=a["n_reps"], n_batches=a["n_batches"], per_batch=a["per_batch"],
                            n_time_bins=a["n_time_bins"], n_census=a.get("n_census", 0),
                            pc_target=a.get("pc_target", 0))
    prob = mc.mc_problem(geometry=mc.MC_GEOM_PULSE, source=0, seeding=a["seeding"], n_bins=a["n_time_bins"],
                         n_batches=a["n_reps"] * a["n_batches"], reserved=0, L=0.0, sigma_t=a["sigma_t"],
                         c=a["c"], n_histories=azurv1_histories(a), seed=a["seed"], stride_q=a["stride_q"],
                         id_offset=a["id_offset"], key=0, tally_offset=a["tally_offset"], box=None,
                         pulse=ctypes.pointer(spec))
    return prob, spec

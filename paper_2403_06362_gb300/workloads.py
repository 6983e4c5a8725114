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

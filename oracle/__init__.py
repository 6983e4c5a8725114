"""ctypes wrapper of the plain C oracle (``mc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check of
``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``.  The product
library never imports this package, and this package never imports it.

Each wrapper follows the paper passage cited in ``mc_oracle.c``: Eq. (1)
(LCG step), Eq. (2) (Brown's skip-ahead), Listing 1 and Eqs. (3)-(5)
(hash seeding), and the Section 5 statistics (batch normality).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mc_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "mc_oracle_box.c"), os.path.join(_HERE, "mc_oracle_azurv1.c"),
         os.path.join(_HERE, "mc_oracle_census.c")]
_LIB = os.path.join(_HERE, "liboracle.so")

NCOUNT = 17
COUNT_NAMES = [
    "source", "flights", "collisions", "absorptions", "scatters", "leak_lo", "leak_hi",
    "draws", "exceed_hist", "exceed_draws", "splits", "roulette_kills", "capped",
    "max_draws", "children", "dropped", "banked",
]
SEED_HASH, SEED_STRIDE, SEED_HASH_HIER = 0, 1, 2
SRC_ISOTROPIC, SRC_BEAM = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -ffp-contract=off, no fast-math)."""
    newest = max(os.path.getmtime(f) for f in _SRCS + [os.path.join(_HERE, "mc_oracle.h")])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11", "-fPIC",
             "-shared", "-Wall", "-o", tmp, *_SRCS, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Lcg(C.Structure):
    _fields_ = [("m", C.c_uint32), ("pad", C.c_uint32), ("g", C.c_uint64), ("c", C.c_uint64)]


BOX_MAX_GROUPS = 8


class BoxProblem(C.Structure):
    _fields_ = [
        ("side", C.c_double), ("inner_lo", C.c_double), ("inner_hi", C.c_double),
        ("sigma_t", C.c_double * 2), ("c", C.c_double * 2),
        ("ww_low", C.c_double * 2), ("ww_high", C.c_double * 2), ("ww_survive", C.c_double * 2),
        ("cdf", ((C.c_double * BOX_MAX_GROUPS) * BOX_MAX_GROUPS) * 2),
        ("n_histories", C.c_uint64), ("seed", C.c_uint64), ("stride_q", C.c_uint64),
        ("id_offset", C.c_uint64), ("key", C.c_uint64), ("tally_offset", C.c_uint64),
        ("n_groups", C.c_uint32), ("mesh", C.c_uint32), ("max_split", C.c_uint32),
        ("n_batches", C.c_uint32), ("seeding", C.c_uint32), ("source", C.c_uint32),
    ]


class Azurv1Problem(C.Structure):
    _fields_ = [
        ("c", C.c_double), ("nu", C.c_double), ("t_end", C.c_double), ("x_half", C.c_double),
        ("sigma_t", C.c_double),
        ("seed", C.c_uint64), ("stride_q", C.c_uint64), ("id_offset", C.c_uint64), ("tally_offset", C.c_uint64),
        ("n_reps", C.c_uint32), ("n_batches", C.c_uint32), ("per_batch", C.c_uint32),
        ("n_time_bins", C.c_uint32), ("seeding", C.c_uint32), ("n_census", C.c_uint32),
        ("pc_target", C.c_uint32), ("pad", C.c_uint32),
    ]


class SlabProblem(C.Structure):
    _fields_ = [
        ("L", C.c_double), ("sigma_t", C.c_double), ("c", C.c_double),
        ("n_histories", C.c_uint64), ("seed", C.c_uint64), ("stride_q", C.c_uint64),
        ("id_offset", C.c_uint64), ("key", C.c_uint64), ("tally_offset", C.c_uint64),
        ("n_bins", C.c_uint32), ("n_batches", C.c_uint32),
        ("source", C.c_uint32), ("seeding", C.c_uint32),
    ]


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            u64, u32, dbl = C.c_uint64, C.c_uint32, C.c_double
            P = C.c_void_p
            L.or_mask.restype = u64; L.or_mask.argtypes = [u32]
            L.or_lcg_next.restype = u64; L.or_lcg_next.argtypes = [u64, u32, u64, u64]
            L.or_u01.restype = dbl; L.or_u01.argtypes = [u64, u32]
            L.or_lcg_skip.restype = u64; L.or_lcg_skip.argtypes = [u64, u64, u32, u64, u64]
            L.or_stride_seed.restype = u64
            L.or_stride_seed.argtypes = [u64, u64, u64, u32, u64, u64]
            L.or_subhash.restype = u64; L.or_subhash.argtypes = [u64]
            L.or_hash.restype = u64; L.or_hash.argtypes = [u64, u64]
            L.or_hash_seed.restype = u64; L.or_hash_seed.argtypes = [u64, u64, u32]
            L.or_seed_hash.restype = None; L.or_seed_hash.argtypes = [u32, u64, u64, u64, P]
            L.or_seed_stride.restype = None
            L.or_seed_stride.argtypes = [u32, u64, u64, u64, u64, u64, u64, P]
            L.or_lcg_draw.restype = None
            L.or_lcg_draw.argtypes = [u32, u64, u64, P, u64, u32, P, P]
            L.or_slab_seed.restype = u64
            L.or_slab_seed.argtypes = [C.POINTER(Lcg), C.POINTER(SlabProblem), u64]
            L.or_batch_of.restype = u64; L.or_batch_of.argtypes = [u64, u64, u32]
            L.or_slab_run.restype = C.c_int
            L.or_slab_run.argtypes = [C.POINTER(Lcg), C.POINTER(SlabProblem), u64, u64, u64,
                                      P, P, P, P, P]
            BP = C.POINTER(BoxProblem)
            L.or_box_seed.restype = u64; L.or_box_seed.argtypes = [C.POINTER(Lcg), BP, u64]
            L.or_box_run.restype = C.c_int
            L.or_box_run.argtypes = [C.POINTER(Lcg), BP, u64, u64, u64, P, P, P, P, P]
            L.or_box_iso_dir.restype = u64; L.or_box_iso_dir.argtypes = [C.POINTER(Lcg), u64, P]
            L.or_box_trace.restype = None; L.or_box_trace.argtypes = [BP, P, P, dbl, dbl, P, P]
            L.or_box_surface_dist.restype = dbl
            L.or_box_surface_dist.argtypes = [BP, P, P, u32, C.POINTER(C.c_int)]
            L.or_box_next_group.restype = u32; L.or_box_next_group.argtypes = [BP, u32, u32, dbl]
            AP = C.POINTER(Azurv1Problem)
            L.or_azurv1_seed.restype = u64; L.or_azurv1_seed.argtypes = [C.POINTER(Lcg), AP, u64]
            L.or_azurv1_run.restype = C.c_int
            L.or_azurv1_run.argtypes = [C.POINTER(Lcg), AP, u64, u64, u64, P, P, P, P]
            L.or_azurv1_census_run.restype = C.c_int
            L.or_azurv1_census_run.argtypes = [C.POINTER(Lcg), AP, u64, u64, u64, P, P, C.c_int, P, P]
            L.or_norm_cdf.restype = dbl; L.or_norm_cdf.argtypes = [dbl]
            L.or_norm_ppf.restype = dbl; L.or_norm_ppf.argtypes = [dbl]
            L.or_shapiro_wilk.restype = C.c_int
            L.or_shapiro_wilk.argtypes = [P, C.c_int, P, P]
            L.or_batch_stats.restype = C.c_int
            L.or_batch_stats.argtypes = [P, u32, u32, P, P, P]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --- Eq. (1), Eq. (2), Listing 1 ------------------------------------------------

def lcg_next(x, m, g, c):
    return int(lib().or_lcg_next(x, m, g, c))


def u01(x, m):
    return float(lib().or_u01(x, m))


def lcg_skip(x0, k, m, g, c):
    return int(lib().or_lcg_skip(x0, k, m, g, c))


def stride_seed(x0, q, k, m, g, c):
    return int(lib().or_stride_seed(x0, q, k, m, g, c))


def subhash(x):
    return int(lib().or_subhash(x))


def hash64(k, s):
    return int(lib().or_hash(k, s))


def hash_seed(k, s, m):
    return int(lib().or_hash_seed(k, s, m))


def seed_hash(m, parent, key_begin, count):
    out = np.empty(count, dtype=np.uint64)
    lib().or_seed_hash(m, parent, key_begin, count, _ptr(out))
    return out


def seed_stride(m, g, c, x0, q, id_begin, count):
    out = np.empty(count, dtype=np.uint64)
    lib().or_seed_stride(m, g, c, x0, q, id_begin, count, _ptr(out))
    return out


def lcg_draw(m, g, c, states, draws, want_u=True, want_digest=True):
    """Returns (final states, u[draws][n] or None, digest[n] or None)."""
    st = np.ascontiguousarray(states, dtype=np.uint64).copy()
    n = st.size
    u = np.empty((draws, n), dtype=np.float64) if want_u else None
    dg = np.empty(n, dtype=np.uint64) if want_digest else None
    lib().or_lcg_draw(m, g, c, _ptr(st), n, draws, _ptr(u), _ptr(dg))
    return st, u, dg


# --- slab transport -------------------------------------------------------------

def slab_tally_size(problems):
    return max(int(p.tally_offset) + int(p.n_batches) * int(p.n_bins) for p in problems)


def slab_run(lcg: Lcg, prob: SlabProblem, id_begin=0, id_end=None, event_cap=2**62,
             tally=None, tally_fp=None, counts=None, per_history=False):
    """Runs histories [id_begin, id_end) of one problem.  Tally arrays are the
    global ones (indexed through prob.tally_offset) and are accumulated into.
    Returns dict(status, tally, tally_fp, counts, hist_state, hist_draws)."""
    if id_end is None:
        id_end = int(prob.n_histories)
    size = int(prob.tally_offset) + int(prob.n_batches) * int(prob.n_bins)
    if tally is None:
        tally = np.zeros(size, dtype=np.int64)
    if tally_fp is None:
        tally_fp = np.zeros(size, dtype=np.float64)
    if counts is None:
        counts = np.zeros(NCOUNT, dtype=np.uint64)
    n = id_end - id_begin
    hs = np.zeros(n, dtype=np.uint64) if per_history else None
    hd = np.zeros(n, dtype=np.uint64) if per_history else None
    st = lib().or_slab_run(C.byref(lcg), C.byref(prob), id_begin, id_end, event_cap,
                           _ptr(tally), _ptr(tally_fp), _ptr(counts), _ptr(hs), _ptr(hd))
    return dict(status=st, tally=tally, tally_fp=tally_fp, counts=counts,
                hist_state=hs, hist_draws=hd)


def slab_run_threaded(lcg: Lcg, prob: SlabProblem, id_begin, id_end, threads, event_cap=2**62):
    """Splits [id_begin, id_end) into `threads` contiguous ranges run on
    Python threads (ctypes releases the GIL), then sums the per-thread
    results.  Used to time the oracle on all host cores."""
    size = int(prob.tally_offset) + int(prob.n_batches) * int(prob.n_bins)
    parts = []
    bounds = np.linspace(id_begin, id_end, threads + 1).astype(np.int64)

    def work(a, b, out):
        out.append(slab_run(lcg, prob, int(a), int(b), event_cap))

    ths = []
    outs = [[] for _ in range(threads)]
    for t in range(threads):
        th = threading.Thread(target=work, args=(bounds[t], bounds[t + 1], outs[t]))
        th.start()
        ths.append(th)
    for th in ths:
        th.join()
    tally = np.zeros(size, dtype=np.int64)
    tally_fp = np.zeros(size, dtype=np.float64)
    counts = np.zeros(NCOUNT, dtype=np.uint64)
    for o in outs:
        parts.append(o[0])
        tally += o[0]["tally"]
        tally_fp += o[0]["tally_fp"]
        c = o[0]["counts"]
        mx = max(int(counts[13]), int(c[13]))
        counts += c
        counts[13] = mx
    return dict(status=max(p["status"] for p in parts), tally=tally, tally_fp=tally_fp,
                counts=counts)


# --- Section 5 statistics -------------------------------------------------------

def norm_cdf(z):
    return float(lib().or_norm_cdf(z))


def norm_ppf(p):
    return float(lib().or_norm_ppf(p))


def shapiro_wilk(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.zeros(1)
    p = np.zeros(1)
    st = lib().or_shapiro_wilk(_ptr(x), x.size, _ptr(w), _ptr(p))
    if st != 0:
        raise ValueError("Shapiro-Wilk needs 3 <= n <= 5000 and nonzero spread")
    return float(w[0]), float(p[0])


def batch_stats(x):
    """x[n_batches][n_points] -> (z[n_batches][n_points], W[n_points], p[n_points])."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    nb, npnt = x.shape
    z = np.zeros_like(x)
    w = np.zeros(npnt)
    p = np.zeros(npnt)
    lib().or_batch_stats(_ptr(x), nb, npnt, _ptr(z), _ptr(w), _ptr(p))
    return z, w, p


def slab_seed(lcg: Lcg, prob: SlabProblem, local_id: int) -> int:
    """Seed of local history `local_id` (Eq. 3 / Eq. 4 / stride X_{Qk})."""
    return int(lib().or_slab_seed(C.byref(lcg), C.byref(prob), local_id))


# --- two-region box (mc_oracle_box.c) --------------------------------------------

def box_run(lcg: Lcg, prob: BoxProblem, id_begin=0, id_end=None, event_cap=2**62, tally=None,
            tally_fp=None, counts=None, per_history=False):
    if id_end is None:
        id_end = int(prob.n_histories)
    nvox = int(prob.mesh) ** 3
    size = int(prob.tally_offset) + int(prob.n_batches) * nvox
    if tally is None:
        tally = np.zeros(size, dtype=np.int64)
    if tally_fp is None:
        tally_fp = np.zeros(size, dtype=np.float64)
    if counts is None:
        counts = np.zeros(NCOUNT, dtype=np.uint64)
    n = id_end - id_begin
    hs = np.zeros(n, dtype=np.uint64) if per_history else None
    hd = np.zeros(n, dtype=np.uint64) if per_history else None
    st = lib().or_box_run(C.byref(lcg), C.byref(prob), id_begin, id_end, event_cap, _ptr(tally),
                          _ptr(tally_fp), _ptr(counts), _ptr(hs), _ptr(hd))
    return dict(status=st, tally=tally, tally_fp=tally_fp, counts=counts, hist_state=hs, hist_draws=hd)


def box_seed(lcg: Lcg, prob: BoxProblem, local_id: int) -> int:
    return int(lib().or_box_seed(C.byref(lcg), C.byref(prob), local_id))


def box_iso_dir(lcg: Lcg, x: int):
    u = np.zeros(3)
    draws = int(lib().or_box_iso_dir(C.byref(lcg), x, _ptr(u)))
    return u, draws


def box_trace(prob: BoxProblem, p, u, L, w=1.0):
    nvox = int(prob.mesh) ** 3
    t64 = np.zeros(nvox, dtype=np.int64)
    tf = np.zeros(nvox)
    p = np.ascontiguousarray(p, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    lib().or_box_trace(C.byref(prob), _ptr(p), _ptr(u), L, w, _ptr(t64), _ptr(tf))
    return t64, tf


def box_surface_dist(prob: BoxProblem, p, u, region):
    p = np.ascontiguousarray(p, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    k = C.c_int(0)
    d = float(lib().or_box_surface_dist(C.byref(prob), _ptr(p), _ptr(u), region, C.byref(k)))
    return d, int(k.value)


def box_next_group(prob: BoxProblem, region: int, g: int, u: float) -> int:
    """The downscatter group the box transport picks for uniform u."""
    return int(lib().or_box_next_group(C.byref(prob), region, g, u))


# --- the paper's supercritical time-dependent problem (mc_oracle_azurv1.c) -------

def azurv1_run(lcg: Lcg, prob: Azurv1Problem, g_begin=0, g_end=None, event_cap=2**62, tally=None,
               counts=None, per_history=False):
    total = int(prob.n_reps) * int(prob.n_batches) * int(prob.per_batch)
    if g_end is None:
        g_end = total
    size = int(prob.tally_offset) + int(prob.n_reps) * int(prob.n_batches) * int(prob.n_time_bins)
    if tally is None:
        tally = np.zeros(size, dtype=np.int64)
    if counts is None:
        counts = np.zeros(NCOUNT, dtype=np.uint64)
    n = g_end - g_begin
    hs = np.zeros(n, dtype=np.uint64) if per_history else None
    hd = np.zeros(n, dtype=np.uint64) if per_history else None
    st = lib().or_azurv1_run(C.byref(lcg), C.byref(prob), g_begin, g_end, event_cap, _ptr(tally),
                             _ptr(counts), _ptr(hs), _ptr(hd))
    return dict(status=st, tally=tally, counts=counts, hist_state=hs, hist_draws=hd)


def azurv1_census_run(lcg: Lcg, prob: Azurv1Problem, g_begin=0, g_end=None, event_cap=2**62, tally=None,
                      counts=None, reverse=False, populations=False):
    """Census phases with population control; g_begin, g_end on group
    boundaries.  populations: also return the particles starting each phase
    and the weight each of them carries, per group ([groups, n_census])."""
    total = int(prob.n_reps) * int(prob.n_batches) * int(prob.per_batch)
    if g_end is None:
        g_end = total
    size = int(prob.tally_offset) + int(prob.n_reps) * int(prob.n_batches) * int(prob.n_time_bins)
    if tally is None:
        tally = np.zeros(size, dtype=np.int64)
    if counts is None:
        counts = np.zeros(NCOUNT, dtype=np.uint64)
    groups = (g_end - g_begin) // int(prob.per_batch)
    pop = np.zeros((groups, int(prob.n_census)), dtype=np.uint64) if populations else None
    wph = np.zeros((groups, int(prob.n_census)), dtype=np.float64) if populations else None
    st = lib().or_azurv1_census_run(C.byref(lcg), C.byref(prob), g_begin, g_end, event_cap, _ptr(tally),
                                    _ptr(counts), 1 if reverse else 0, _ptr(pop), _ptr(wph))
    return dict(status=st, tally=tally, counts=counts, populations=pop, weights=wph)


def azurv1_seed(lcg: Lcg, prob: Azurv1Problem, g: int) -> int:
    return int(lib().or_azurv1_seed(C.byref(lcg), C.byref(prob), g))

"""ctypes binding of libmc (``include/mc.h``): structures and the C entry
points, one Python function per C function with the same name.

Marshalling only: device buffers are passed as raw pointers taken from torch
tensors (``tensor.data_ptr()``), streams as ``torch.cuda.Stream.cuda_stream``
handles.  Every computation happens in libmc's CUDA kernels; a missing or
stale library is an ImportError, never a fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmc.so")

MC_OK, MC_ERR_ARG, MC_ERR_CUDA, MC_ERR_OVERFLOW = 0, -1, -2, -3
MC_ERR_EVENT_CAP, MC_ERR_TIMEOUT, MC_ERR_CAPACITY, MC_ERR_STATE = -4, -5, -6, -7
MC_SEED_HASH, MC_SEED_STRIDE, MC_SEED_HASH_HIER = 0, 1, 2
MC_SRC_ISOTROPIC, MC_SRC_BEAM = 0, 1
MC_GEOM_SLAB, MC_GEOM_BOX, MC_GEOM_PULSE = 0, 1, 2
MC_FP64, MC_FP32_GUARDED = 0, 1
MC_SCHED_HISTORY, MC_SCHED_EVENT, MC_SCHED_AUTO = 0, 1, 2
MC_NCOUNT = 17
MC_BOX_MAX_GROUPS = 8
COUNT_NAMES = [
    "source", "flights", "collisions", "absorptions", "scatters", "leak_lo", "leak_hi",
    "draws", "exceed_hist", "exceed_draws", "splits", "roulette_kills", "capped",
    "max_draws", "children", "dropped", "banked",
]

EXPORTED = [
    "mc_last_error", "mc_ctx_create", "mc_ctx_destroy", "mc_seed_hash", "mc_seed_stride",
    "mc_lcg_draw", "mc_transport_run", "mc_tally_read", "mc_hash64", "mc_normality",
    "mc_transport_run_static", "mc_autotune", "mc_log1m", "mc_log1m_device", "mc_recip_rn",
    "mc_two_u_minus_1", "mc_recip_rn_device", "mc_llrint_nonneg", "mc_d_lt", "mc_mul_small",
    "mc_ctx_set_limits", "mc_ctx_get_limits", "mc_lcg_draw_host",
]


class McError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libmc status {status}: {msg}")
        self.status = status


class mc_lcg(C.Structure):
    _fields_ = [("m", C.c_uint32), ("reserved", C.c_uint32), ("g", C.c_uint64), ("c", C.c_uint64)]


class mc_seed_spec(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("reserved", C.c_uint32), ("seed", C.c_uint64),
                ("stride_q", C.c_uint64), ("key", C.c_uint64)]


_G = MC_BOX_MAX_GROUPS


class mc_box_spec(C.Structure):
    _fields_ = [
        ("side", C.c_double), ("inner_lo", C.c_double), ("inner_hi", C.c_double),
        ("sigma_t", C.c_double * 2), ("c", C.c_double * 2),
        ("ww_low", C.c_double * 2), ("ww_high", C.c_double * 2), ("ww_survive", C.c_double * 2),
        ("scatter_cdf", ((C.c_double * _G) * _G) * 2),
        ("n_groups", C.c_uint32), ("mesh", C.c_uint32), ("max_split", C.c_uint32),
        ("reserved", C.c_uint32),
    ]


class mc_pulse_spec(C.Structure):
    _fields_ = [
        ("c", C.c_double), ("nu", C.c_double), ("t_end", C.c_double), ("x_half", C.c_double),
        ("sigma_t", C.c_double), ("n_reps", C.c_uint32), ("n_batches", C.c_uint32),
        ("per_batch", C.c_uint32), ("n_time_bins", C.c_uint32), ("n_census", C.c_uint32),
        ("pc_target", C.c_uint32),
    ]


class mc_problem(C.Structure):
    _fields_ = [
        ("geometry", C.c_uint32), ("source", C.c_uint32), ("seeding", C.c_uint32),
        ("n_bins", C.c_uint32), ("n_batches", C.c_uint32), ("reserved", C.c_uint32),
        ("L", C.c_double), ("sigma_t", C.c_double), ("c", C.c_double),
        ("n_histories", C.c_uint64), ("seed", C.c_uint64), ("stride_q", C.c_uint64),
        ("id_offset", C.c_uint64), ("key", C.c_uint64), ("tally_offset", C.c_uint64),
        ("box", C.POINTER(mc_box_spec)), ("pulse", C.POINTER(mc_pulse_spec)),
    ]


class mc_run_config(C.Structure):
    _fields_ = [
        ("schedule", C.c_uint32), ("precision", C.c_uint32), ("block", C.c_uint32),
        ("chunk", C.c_uint32), ("blocks_per_sm", C.c_uint32), ("use_graph", C.c_uint32),
        ("accumulate", C.c_uint32), ("tally_mode", C.c_uint32),
        ("event_cap", C.c_uint64), ("range_begin", C.c_uint64), ("range_end", C.c_uint64),
        ("stack_depth", C.c_uint32), ("tally_atomics", C.c_uint32),
    ]


class mc_limits(C.Structure):
    _fields_ = [
        ("pool_lock_attempts", C.c_uint32), ("box_generations", C.c_uint32),
        ("pulse_generations", C.c_uint32), ("reserved", C.c_uint32), ("event_iterations", C.c_uint64),
    ]


class mc_tally(C.Structure):
    _fields_ = [
        ("d_bins", C.c_void_p), ("n_slots", C.c_uint64), ("d_counts", C.c_void_p),
        ("d_hist_state", C.c_void_p), ("d_hist_draws", C.c_void_p),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`"
            " (libmc has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    u32, u64, i32, P, dbl = C.c_uint32, C.c_uint64, C.c_int, C.c_void_p, C.c_double
    sig = {
        "mc_last_error": (C.c_char_p, []),
        "mc_ctx_create": (i32, [C.POINTER(C.c_void_p), i32]),
        "mc_ctx_destroy": (None, [P]),
        "mc_ctx_set_limits": (i32, [P, C.POINTER(mc_limits)]),
        "mc_ctx_get_limits": (i32, [P, C.POINTER(mc_limits)]),
        "mc_seed_hash": (i32, [P, C.POINTER(mc_lcg), u64, u64, u64, P, P]),
        "mc_seed_stride": (i32, [P, C.POINTER(mc_lcg), u64, u64, u64, u64, P, P]),
        "mc_lcg_draw": (i32, [P, C.POINTER(mc_lcg), C.POINTER(mc_seed_spec), u64, P, u64, u32, P, P, P]),
        "mc_lcg_draw_host": (i32, [P, C.POINTER(mc_lcg), C.POINTER(mc_seed_spec), u64, P, u64, u32, P, P]),
        "mc_transport_run": (i32, [P, C.POINTER(mc_lcg), C.POINTER(mc_problem), u32,
                                   C.POINTER(mc_run_config), C.POINTER(mc_tally), P]),
        "mc_tally_read": (i32, [P, C.POINTER(mc_problem), u32, C.POINTER(mc_tally), P, P, P, P, P, P]),
        "mc_hash64": (u64, [u64, u64]),
        "mc_normality": (i32, [P, u32, u32, P, P, P]),
        "mc_log1m": (dbl, [dbl]),
        "mc_log1m_device": (i32, [P, P, u64, i32, P]),
        "mc_recip_rn": (dbl, [dbl]),
        "mc_two_u_minus_1": (dbl, [u64]),
        "mc_recip_rn_device": (i32, [P, P, u64, i32, P]),
        "mc_llrint_nonneg": (C.c_longlong, [dbl]),
        "mc_d_lt": (i32, [dbl, dbl]),
        "mc_mul_small": (dbl, [u32, dbl]),
        "mc_autotune": (i32, [P, C.POINTER(mc_lcg), C.POINTER(mc_problem), u32, C.POINTER(mc_run_config),
                              C.POINTER(mc_tally), C.POINTER(mc_run_config), C.POINTER(C.c_float), P]),
        "mc_transport_run_static": (i32, [C.POINTER(mc_lcg), C.POINTER(mc_problem), u32,
                                          C.POINTER(mc_run_config), C.POINTER(mc_tally), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = None


def lib():
    """The loaded libmc (loaded on first use; ImportError if it is missing)."""
    global _LIB
    if _LIB is None:
        _LIB = _load()
    return _LIB


def last_error() -> str:
    return lib().mc_last_error().decode(errors="replace")


def check(status: int) -> int:
    if status != MC_OK:
        raise McError(status, last_error())
    return status

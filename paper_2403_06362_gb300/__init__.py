"""GB300-native hash- and stride-seeded LCG streams and Monte Carlo transport.

Python face of libmc (``include/mc.h``).  Each ``mc_*`` function below calls
the C entry point of the same name; arguments are marshalled (torch device
tensors become raw pointers, torch streams become ``cudaStream_t`` handles)
and nothing else happens here: seeding, draws, transport and tallies all run
in libmc's CUDA kernels.  The method is that of Cuneo & Variansyah, "An
Alternative to Stride-Based RNG for Monte Carlo Transport" (arXiv
2403.06362): Eq. (1) LCG, Eq. (2) stride skip-ahead, Listing 1 and
Eqs. (3)-(5) hash seed splitting.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import _ffi
from ._ffi import (  # noqa: F401  (re-exported names)
    COUNT_NAMES, MC_FP32_GUARDED, MC_FP64, MC_GEOM_BOX, MC_GEOM_PULSE, MC_GEOM_SLAB, MC_NCOUNT,
    MC_SCHED_AUTO, mc_pulse_spec,
    MC_SCHED_EVENT, MC_SCHED_HISTORY, MC_SEED_HASH, MC_SEED_HASH_HIER, MC_SEED_STRIDE,
    MC_SRC_BEAM, MC_SRC_ISOTROPIC, McError, mc_box_spec, mc_lcg, mc_limits, mc_problem, mc_run_config,
    mc_seed_spec, mc_tally,
)

LIB_PATH = _ffi.LIB_PATH


def lib():
    """libmc, loaded on first use; raises ImportError when it has not been built."""
    return _ffi.lib()


def _ptr(t) -> Optional[int]:
    """Raw pointer of a torch tensor (or None / int passthrough)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("libmc needs contiguous buffers")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_lcg(m=63, g=2806196910506780709, c=1) -> mc_lcg:
    return mc_lcg(m=m, reserved=0, g=g, c=c)


class Context:
    """Owns an mc_ctx (library scratch on one device)."""

    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _ffi.check(lib().mc_ctx_create(C.byref(h), device))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().mc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mc_ctx_create(device: int = 0) -> Context:
    return Context(device)


def mc_ctx_destroy(ctx: Context) -> None:
    ctx.close()


def mc_ctx_set_limits(ctx: Context, limits: Optional[mc_limits] = None) -> None:
    """Bounds on the waits of a run under ctx (None restores the defaults)."""
    _ffi.check(lib().mc_ctx_set_limits(ctx.handle, C.byref(limits) if limits is not None else None))


def mc_ctx_get_limits(ctx: Context) -> mc_limits:
    out = mc_limits()
    _ffi.check(lib().mc_ctx_get_limits(ctx.handle, C.byref(out)))
    return out


def mc_last_error() -> str:
    return _ffi.last_error()


def mc_hash64(k: int, s: int) -> int:
    return int(lib().mc_hash64(k, s))


def mc_log1m(u: float) -> float:
    """ln(1 - u) by the fp64 flight logarithm, evaluated on the host."""
    return float(lib().mc_log1m(float(u)))


def mc_log1m_device(d_u, d_out, which=0, stream=None):
    """d_out = ln(1 - d_u) on the device: which 0 = the flight logarithm,
    1 = the CUDA library's log (fp64 tensors of equal length)."""
    return _ffi.check(lib().mc_log1m_device(_ptr(d_u), _ptr(d_out), d_u.numel(), which, _stream(stream)))


def mc_recip_rn(y: float) -> float:
    """1/y rounded to nearest, by the integer-pipe reciprocal (host evaluation)."""
    return float(lib().mc_recip_rn(float(y)))


def mc_two_u_minus_1(n: int) -> float:
    """2u - 1 for u = n 2^-53, assembled from integer operations (host evaluation)."""
    return float(lib().mc_two_u_minus_1(int(n)))


def mc_mul_small(j: int, h: float) -> float:
    """RN(j h) for a small integer j, assembled from integer operations (host evaluation)."""
    return float(lib().mc_mul_small(int(j), float(h)))


def mc_recip_rn_device(d_y, d_out, which=0, stream=None):
    """d_out = 1/d_y on the device: which 0 = the integer-pipe reciprocal,
    1 = the CUDA division (fp64 tensors of equal length)."""
    return _ffi.check(lib().mc_recip_rn_device(_ptr(d_y), _ptr(d_out), d_y.numel(), which, _stream(stream)))


def mc_seed_hash(ctx, lcg, parent_seed, key_begin, count, d_states, stream=None):
    return _ffi.check(lib().mc_seed_hash(ctx.handle, C.byref(lcg), parent_seed, key_begin, count,
                                       _ptr(d_states), _stream(stream)))


def mc_seed_stride(ctx, lcg, x0, stride_q, id_begin, count, d_states, stream=None):
    return _ffi.check(lib().mc_seed_stride(ctx.handle, C.byref(lcg), x0, stride_q, id_begin, count,
                                         _ptr(d_states), _stream(stream)))


def mc_lcg_draw(ctx, lcg, seed, id_begin, d_states, n_streams, draws, d_u=None, d_digest=None,
                stream=None):
    sp = C.byref(seed) if seed is not None else None
    return _ffi.check(lib().mc_lcg_draw(ctx.handle, C.byref(lcg), sp, id_begin, _ptr(d_states),
                                      n_streams, draws, _ptr(d_u), _ptr(d_digest), _stream(stream)))


def _host_ptr(a) -> Optional[int]:
    """Raw pointer of a host buffer: a torch CPU tensor or a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("mc_lcg_draw_host needs contiguous host buffers")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("mc_lcg_draw_host needs contiguous host buffers")
    return a.ctypes.data


def mc_lcg_draw_host(ctx, lcg, seed, id_begin, h_states, n_streams, draws, h_digest=None, stream=None):
    """mc_lcg_draw on host buffers (uint64 / int64 arrays or CPU tensors;
    page-locked ones let the library overlap copies and kernels)."""
    sp = C.byref(seed) if seed is not None else None
    return _ffi.check(lib().mc_lcg_draw_host(ctx.handle, C.byref(lcg), sp, id_begin, _host_ptr(h_states),
                                           n_streams, draws, _host_ptr(h_digest), _stream(stream)))


def problem_array(problems: Sequence[mc_problem]):
    arr = (mc_problem * len(problems))(*problems)
    return arr


def mc_transport_run(ctx, lcg, problems, config, tally, stream=None):
    arr = problems if isinstance(problems, C.Array) else problem_array(problems)
    return _ffi.check(lib().mc_transport_run(ctx.handle, C.byref(lcg), arr, len(arr), C.byref(config),
                                           C.byref(tally), _stream(stream)))


def mc_autotune(ctx, lcg, problems, base, tally, stream=None):
    """Returns (best mc_run_config, its time in ms on the tuning sample)."""
    arr = problems if isinstance(problems, C.Array) else problem_array(problems)
    best = mc_run_config()
    ms = C.c_float(0.0)
    _ffi.check(lib().mc_autotune(ctx.handle, C.byref(lcg), arr, len(arr), C.byref(base), C.byref(tally),
                                 C.byref(best), C.byref(ms), _stream(stream)))
    return best, float(ms.value)


def mc_transport_run_static(lcg, problems, config, tally, stream=None):
    """mc_transport_run without a context: scratch lives in a fixed device
    array inside libmc (for callers that cannot allocate device memory)."""
    arr = problems if isinstance(problems, C.Array) else problem_array(problems)
    return _ffi.check(lib().mc_transport_run_static(C.byref(lcg), arr, len(arr), C.byref(config),
                                                    C.byref(tally), _stream(stream)))


@dataclass
class TallyRead:
    status: int
    flux: np.ndarray
    rel_err: np.ndarray
    batch: np.ndarray
    raw: np.ndarray
    counts: dict


def mc_tally_read(ctx, problems, index, tally, stream=None, check=True) -> TallyRead:
    arr = problems if isinstance(problems, C.Array) else problem_array(problems)
    p = arr[index]
    nb, nbat = int(p.n_bins), int(p.n_batches)
    flux = np.zeros(nb)
    rel = np.zeros(nb)
    batch = np.zeros((nbat, nb))
    raw = np.zeros((nbat, nb), dtype=np.int64)
    cnt = np.zeros(MC_NCOUNT, dtype=np.uint64)
    P = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    st = lib().mc_tally_read(ctx.handle, arr, index, C.byref(tally), P(flux), P(rel), P(batch), P(raw),
                           P(cnt), _stream(stream))
    if check and st not in (_ffi.MC_OK,):
        raise McError(st, _ffi.last_error())
    return TallyRead(st, flux, rel, batch, raw, dict(zip(COUNT_NAMES, (int(v) for v in cnt))))


def mc_normality(x: np.ndarray):
    """x[n_batches][n_points] -> (z, W, p) of the Section 5 procedure."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    nb, npnt = x.shape
    z = np.zeros_like(x)
    w = np.zeros(npnt)
    p = np.zeros(npnt)
    P = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    st = lib().mc_normality(P(x), nb, npnt, P(z), P(w), P(p))
    if st != 0:
        raise McError(st, "mc_normality: n_batches outside [3, 5000] or a point without spread")
    return z, w, p


class Tally:
    """Device buffers of an mc_tally, allocated with torch (plumbing only)."""

    def __init__(self, n_slots: int, n_problems: int, n_histories: int = 0, device="cuda"):
        import torch
        self.bins = torch.zeros(n_slots, dtype=torch.int64, device=device)
        self.counts = torch.zeros(n_problems * MC_NCOUNT, dtype=torch.int64, device=device)
        self.hist_state = (torch.zeros(n_histories, dtype=torch.int64, device=device)
                           if n_histories else None)
        self.hist_draws = (torch.zeros(n_histories, dtype=torch.int64, device=device)
                           if n_histories else None)
        self.c = mc_tally(d_bins=_ptr(self.bins), n_slots=n_slots, d_counts=_ptr(self.counts),
                          d_hist_state=_ptr(self.hist_state), d_hist_draws=_ptr(self.hist_draws))

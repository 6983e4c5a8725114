"""The C-ABI library builds, loads and exports every entry point that
include/mc.h declares; host-side argument checks and host helpers behave
(no device compute is called here)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mc.h")


@pytest.fixture(scope="session")
def mc():
    from paper_2403_06362_gb300 import _build
    _build.build()
    import paper_2403_06362_gb300 as mc
    mc.lib()
    return mc


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"MC_API\s+[\w\s\*]+?\b(mc_\w+)\s*\(", text)


def test_header_declares_the_five_calls():
    names = set(declared_functions())
    for n in ("mc_seed_hash", "mc_seed_stride", "mc_lcg_draw", "mc_transport_run", "mc_tally_read"):
        assert n in names


def test_every_declared_symbol_is_exported(mc):
    out = subprocess.run(["nm", "-D", "--defined-only", mc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(mc_\w+)", out))
    declared = set(declared_functions())
    assert declared <= exported, declared - exported
    lib = mc.lib()
    for n in declared:
        assert getattr(lib, n) is not None


def test_argument_errors_are_reported_without_a_gpu(mc):
    lib = mc.lib()
    lcg = mc.make_lcg()
    assert lib.mc_seed_hash(None, C.byref(lcg), 42, 0, 10, None, None) == mc._ffi.MC_ERR_ARG
    assert "ctx" in mc.mc_last_error()
    bad = mc.make_lcg(g=2)
    assert lib.mc_seed_stride(C.c_void_p(1), C.byref(bad), 1, 3, 0, 10, C.c_void_p(16), None) == mc._ffi.MC_ERR_ARG
    assert "odd" in mc.mc_last_error()
    bad_m = mc.make_lcg(m=65)
    assert lib.mc_lcg_draw(C.c_void_p(1), C.byref(bad_m), None, 0, C.c_void_p(16), 4, 4, None, None,
                           None) == mc._ffi.MC_ERR_ARG
    # unaligned state buffer
    assert lib.mc_seed_hash(C.c_void_p(1), C.byref(lcg), 42, 0, 10, C.c_void_p(12), None) == mc._ffi.MC_ERR_ARG
    # transport: no problems
    cfg = mc.mc_run_config()
    t = mc.mc_tally()
    assert lib.mc_transport_run(C.c_void_p(1), C.byref(lcg), None, 0, C.byref(cfg), C.byref(t), None) \
        == mc._ffi.MC_ERR_ARG
    # wait bounds: no context
    lim = mc.mc_limits()
    assert lib.mc_ctx_set_limits(None, C.byref(lim)) == mc._ffi.MC_ERR_ARG
    assert lib.mc_ctx_get_limits(None, C.byref(lim)) == mc._ffi.MC_ERR_ARG


def test_host_hash_matches_oracle(mc, oracle):
    rng = np.random.default_rng(3)
    for k, s in [(0, 42), (1, 42), (2**26 - 1, 42)] + [tuple(int(v) for v in rng.integers(0, 2**62, 2))
                                                       for _ in range(100)]:
        assert mc.mc_hash64(k, s) == oracle.hash64(k, s)


def test_host_normality_matches_oracle(mc, oracle):
    rng = np.random.default_rng(4)
    for nb in (3, 4, 5, 6, 10, 11, 12, 20, 1000):
        x = rng.normal(size=(nb, 5))
        z, w, p = mc.mc_normality(x)
        oz, ow, op = oracle.batch_stats(x)
        assert np.allclose(z, oz, rtol=1e-12, atol=1e-14)
        assert np.allclose(w, ow, rtol=1e-12, atol=0)
        assert np.allclose(p, op, rtol=1e-9, atol=1e-15)
    with pytest.raises(mc.McError):
        mc.mc_normality(np.zeros((2, 3)))

"""The integer-pipe reciprocal on the device: the same bits as the host copy
(tests/test_fp_exact.py checks that one against IEEE division) and as the
CUDA fp64 division, over 2^22 random doubles and the edge cases."""
import numpy as np
import pytest
import torch

import paper_2403_06362_gb300 as mc

pytestmark = pytest.mark.gpu


def inputs(n):
    rng = np.random.default_rng(105)
    e = rng.integers(1, 2044, size=n, dtype=np.uint64)
    m = rng.integers(0, 2**52, size=n, dtype=np.uint64)
    b = (e << np.uint64(52)) | m
    b[: n // 2] |= np.uint64(1) << np.uint64(63)  # half negative
    edges = np.array([1.0, -1.0, 2.0**-1000, 2.0**1000, 1.0 + 2.0**-52, 2.0 - 2.0**-52, 5e-324, 1.7e308],
                     dtype=np.float64).view(np.uint64)
    return np.concatenate([b, edges]).view(np.float64)


def on_device(y, which):
    dy = torch.from_numpy(y).cuda()
    out = torch.empty_like(dy)
    mc.mc_recip_rn_device(dy, out, which)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_device_reciprocal_matches_cuda_division_and_host():
    y = inputs(1 << 22)
    ours, lib = on_device(y, 0), on_device(y, 1)
    assert np.array_equal(ours.view(np.uint64), lib.view(np.uint64))
    idx = np.random.default_rng(1).choice(y.size, 5000, replace=False)
    host = np.array([mc.mc_recip_rn(float(v)) for v in y[idx]])
    assert np.array_equal(ours[idx].view(np.uint64), host.view(np.uint64))

"""The fp64 flight logarithm on the device: the same bits as the host copy
(whose accuracy tests/test_log.py measures), and within one ulp of the CUDA
library's log, over 2^22 uniforms of the LCG and the edge cases."""
import math

import numpy as np
import pytest
import torch

import paper_2403_06362_gb300 as mc

pytestmark = pytest.mark.gpu


def uniforms(n):
    rng = np.random.default_rng(2403)
    k = rng.integers(0, 2**53, size=n, dtype=np.uint64)
    small = rng.integers(1, 2**40, size=n // 8, dtype=np.uint64) >> rng.integers(0, 40, size=n // 8).astype(np.uint64)
    edges = np.array([0, 1, 2**45 - 1, 2**45, 2**45 + 1, 2**52, 2**53 - 1], dtype=np.uint64)
    return np.concatenate([k, small, edges]).astype(np.float64) * 2.0**-53


def on_device(u, which):
    du = torch.from_numpy(u).cuda()
    out = torch.empty_like(du)
    mc.mc_log1m_device(du, out, which)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_device_matches_host_bits():
    u = uniforms(1 << 22)
    dev = on_device(u, 0)
    idx = np.random.default_rng(1).choice(u.size, 20000, replace=False)
    idx = np.concatenate([idx, np.arange(u.size - 7, u.size)])
    host = np.array([mc.mc_log1m(float(u[i])) for i in idx])
    assert np.array_equal(dev[idx].view(np.uint64), host.view(np.uint64))


def test_within_one_ulp_of_cuda_log():
    u = uniforms(1 << 22)
    ours, lib = on_device(u, 0), on_device(u, 1)
    diff = np.abs(ours.view(np.int64) - lib.view(np.int64))
    assert diff.max() <= 1
    assert (diff == 0).mean() > 0.95
    assert ours[-7] == 0.0 and ours[-1] == math.log(2.0**-53)


def test_rejects_bad_arguments():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(mc.McError):
        mc.mc_log1m_device(x, x, which=2)

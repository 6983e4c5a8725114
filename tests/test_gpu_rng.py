"""GPU parity of seeding and draws (mc_seed_hash, mc_seed_stride,
mc_lcg_draw) against the oracle: bit-exact states, uniforms and digests, at
small ragged sizes, edge cases, and the full 2^26-stream microbenchmark
(in the launch configuration the benchmark times) on sampled outputs."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W

pytestmark = pytest.mark.gpu

M, G, CC, Q = W.LCG_M, W.LCG_G, W.LCG_C, W.STRIDE_Q


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import _build
    _build.build()
    ctx = mc.Context(0)
    yield mc, ctx, torch
    torch.cuda.synchronize()
    ctx.close()


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def dev_u64(torch, n, offset=0):
    buf = torch.zeros(n + offset, dtype=torch.int64, device="cuda")
    return buf[offset:], buf


@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 1000, 4097, 100_003])
@pytest.mark.parametrize("offset", [0, 1])
def test_seed_hash_small(env, oracle, n, offset):
    mc, ctx, torch = env
    v, _ = dev_u64(torch, n, offset)  # offset 1: 8-byte aligned, not 16
    mc.mc_seed_hash(ctx, mc.make_lcg(), 42, 17, n, v if n else None)
    if n:
        assert np.array_equal(u64(v), oracle.seed_hash(M, 42, 17, n))


@pytest.mark.parametrize("n", [1, 2, 3, 33, 4097, 100_003])
@pytest.mark.parametrize("offset", [0, 1])
def test_seed_stride_small(env, oracle, n, offset):
    mc, ctx, torch = env
    v, _ = dev_u64(torch, n, offset)
    mc.mc_seed_stride(ctx, mc.make_lcg(), 1, Q, 5, n, v)
    assert np.array_equal(u64(v), oracle.seed_stride(M, G, CC, 1, Q, 5, n))


@pytest.mark.parametrize("m", [64, 62, 53, 33, 20])
def test_other_widths(env, oracle, m):
    mc, ctx, torch = env
    n, draws = 3001, 9
    g, c = (G, CC)
    lcg = mc.make_lcg(m=m, g=g, c=c)
    v, _ = dev_u64(torch, n)
    mc.mc_seed_hash(ctx, lcg, 7, 0, n, v)
    assert np.array_equal(u64(v), oracle.seed_hash(m, 7, 0, n))
    mc.mc_seed_stride(ctx, lcg, 3, 1000, 2**40, n, v)
    seeds = oracle.seed_stride(m, g, c, 3, 1000, 2**40, n)
    assert np.array_equal(u64(v), seeds)
    u = torch.empty(draws * n, dtype=torch.float64, device="cuda")
    dg = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, lcg, None, 0, v, n, draws, u, dg)
    o_st, o_u, o_dg = oracle.lcg_draw(m, g, c, seeds, draws)
    assert np.array_equal(u64(v), o_st)
    assert np.array_equal(u.cpu().numpy().reshape(draws, n), o_u)
    assert np.array_equal(u64(dg), o_dg)


@pytest.mark.parametrize("draws", [0, 1, 7, 8, 9, 64, 65])
@pytest.mark.parametrize("n", [1, 777, 20_001])
def test_draws_loaded_states(env, oracle, draws, n):
    mc, ctx, torch = env
    seeds = oracle.seed_hash(M, 42, 1000, n)
    v = torch.from_numpy(seeds.view(np.int64).copy()).cuda()
    u = torch.full((max(draws, 1) * n,), -1.0, dtype=torch.float64, device="cuda")
    dg = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), None, 0, v, n, draws, u, dg)
    o_st, o_u, o_dg = oracle.lcg_draw(M, G, CC, seeds, draws)
    assert np.array_equal(u64(v), o_st)
    assert np.array_equal(u64(dg), o_dg)
    if draws:
        assert np.array_equal(u.cpu().numpy().reshape(draws, n), o_u)


@pytest.mark.parametrize("mode", ["hash", "stride", "hier"])
def test_fused_seed_and_draw(env, oracle, mode):
    mc, ctx, torch = env
    n, draws, id0 = 50_001, 64, 123
    if mode == "stride":
        spec = mc.mc_seed_spec(mode=mc.MC_SEED_STRIDE, seed=1, stride_q=Q)
        seeds = oracle.seed_stride(M, G, CC, 1, Q, id0, n)
    elif mode == "hash":
        spec = mc.mc_seed_spec(mode=mc.MC_SEED_HASH, seed=42)
        seeds = oracle.seed_hash(M, 42, id0, n)
    else:
        spec = mc.mc_seed_spec(mode=mc.MC_SEED_HASH_HIER, seed=42, key=9)
        seeds = oracle.seed_hash(M, oracle.hash64(9, 42), id0, n)
    v, _ = dev_u64(torch, n)
    u = torch.empty(draws * n, dtype=torch.float64, device="cuda")
    dg = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), spec, id0, v, n, draws, u, dg)
    o_st, o_u, o_dg = oracle.lcg_draw(M, G, CC, seeds, draws)
    assert np.array_equal(u64(v), o_st)
    assert np.array_equal(u.cpu().numpy().reshape(draws, n), o_u)
    assert np.array_equal(u64(dg), o_dg)
    # digest only, no states (the benchmark's form)
    dg2 = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), spec, id0, None, n, draws, None, dg2)
    assert np.array_equal(u64(dg2), o_dg)


def test_uniform_range_and_exactness(env, oracle):
    mc, ctx, torch = env
    # states whose top bits are zero exercise the rare conversion branches
    special = np.array([0, 1, 1023, 1024, 2**32, 2**42 - 1, 2**42, 2**62, 2**63 - 1,
                        2**43 + 5, 2**52], dtype=np.uint64)
    n = special.size
    v = torch.from_numpy(special.view(np.int64).copy()).cuda()
    # one draw from state y gives u01(g*y + c); pick y = g^-1 (x - c) so the
    # first state is x itself
    ginv = pow(G, -1, 2**63)
    pre = np.array([((int(x) - CC) * ginv) % 2**63 for x in special], dtype=np.uint64)
    v = torch.from_numpy(pre.view(np.int64).copy()).cuda()
    u = torch.empty(n, dtype=torch.float64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), None, 0, v, n, 1, u, None)
    assert np.array_equal(u64(v), special)
    got = u.cpu().numpy()
    exp = np.array([oracle.u01(int(x), 63) for x in special])
    assert np.array_equal(got, exp)
    assert got.min() >= 0.0 and got.max() < 1.0


def test_full_microbench_sampled(env, oracle):
    """2^26 streams x 64 draws, hash and stride, in the benchmark's launch
    configuration (fused seeding, digest + final state); every seed of the
    hash mode is checked, and sampled streams of both modes bit for bit."""
    mc, ctx, torch = env
    n, draws = 2**26, 64
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([np.arange(4096), n - 1 - np.arange(4096),
                                       rng.integers(0, n, 20_000)]))
    st = torch.empty(n, dtype=torch.int64, device="cuda")
    dg = torch.empty(n, dtype=torch.int64, device="cuda")
    seeds_dev = torch.empty(n, dtype=torch.int64, device="cuda")
    for mode in ("hash", "stride"):
        if mode == "hash":
            spec = mc.mc_seed_spec(mode=mc.MC_SEED_HASH, seed=42)
            mc.mc_seed_hash(ctx, mc.make_lcg(), 42, 0, n, seeds_dev)
            all_seeds = oracle.seed_hash(M, 42, 0, n)
            assert np.array_equal(u64(seeds_dev), all_seeds)
            seeds = all_seeds[sample]
        else:
            spec = mc.mc_seed_spec(mode=mc.MC_SEED_STRIDE, seed=1, stride_q=Q)
            mc.mc_seed_stride(ctx, mc.make_lcg(), 1, Q, 0, n, seeds_dev)
            seeds = np.array([oracle.stride_seed(1, Q, int(k), M, G, CC) for k in sample], dtype=np.uint64)
            assert np.array_equal(u64(seeds_dev)[sample], seeds)
        mc.mc_lcg_draw(ctx, mc.make_lcg(), spec, 0, st, n, draws, None, dg)
        o_st, _, o_dg = oracle.lcg_draw(M, G, CC, seeds, draws, want_u=False)
        assert np.array_equal(u64(st)[sample], o_st)
        assert np.array_equal(u64(dg)[sample], o_dg)
        # unfused path agrees everywhere with the fused one
        dg2 = torch.empty(n, dtype=torch.int64, device="cuda")
        mc.mc_lcg_draw(ctx, mc.make_lcg(), None, 0, seeds_dev, n, draws, None, dg2)
        assert torch.equal(dg, dg2) and torch.equal(st, seeds_dev)


@pytest.mark.parametrize("draws", [0, 1, 2, 15, 16, 17, 63, 64, 65, 130])
@pytest.mark.parametrize("n", [1, 2, 3, 1001, 65_537])
def test_digest_only_kernel(env, oracle, draws, n):
    # the integer-issue-bound form (no uniforms stored): two streams per
    # thread, compile-time and run-time draw counts, odd stream counts
    mc, ctx, torch = env
    seeds = oracle.seed_hash(M, 7, 99, n)
    v = torch.from_numpy(seeds.view(np.int64).copy()).cuda()
    dg = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), None, 0, v, n, draws, None, dg)
    o_st, _, o_dg = oracle.lcg_draw(M, G, CC, seeds, draws, want_u=False)
    assert np.array_equal(u64(v), o_st)
    assert np.array_equal(u64(dg), o_dg)


@pytest.mark.parametrize("draws", [5, 64, 65])
def test_digest_kernel_rare_conversion_path(env, oracle, draws):
    # first states below 2^31 (high word of the doubled state zero) force the
    # exact redo; those from 2^31 up take the branch-free path with
    # normalising shifts up to 31
    mc, ctx, torch = env
    special = np.array([0, 1, 1023, 1024, 2**31 - 1, 2**31, 2**31 + 1, 2**32 - 1, 2**32, 2**33 - 1,
                        2**42 - 1, 2**42, 2**43 + 5, 2**52, 2**62, 2**63 - 1], dtype=np.uint64)
    ginv = pow(G, -1, 2**63)
    pre = np.array([((int(x) - CC) * ginv) % 2**63 for x in special], dtype=np.uint64)
    pre = np.concatenate([pre, oracle.seed_hash(M, 1, 0, 101)])
    v = torch.from_numpy(pre.view(np.int64).copy()).cuda()
    dg = torch.empty(pre.size, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), None, 0, v, pre.size, draws, None, dg)
    o_st, _, o_dg = oracle.lcg_draw(M, G, CC, pre, draws, want_u=False)
    assert np.array_equal(u64(v), o_st)
    assert np.array_equal(u64(dg), o_dg)


def test_digest_kernel_long_streams(env, oracle):
    # run-time draw count far beyond what one fp32 count sum holds exactly
    # (the kernel folds it into an integer every 16 draws)
    mc, ctx, torch = env
    n, draws = 5, 600_001
    seeds = oracle.seed_hash(M, 3, 0, n)
    v = torch.from_numpy(seeds.view(np.int64).copy()).cuda()
    dg = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), None, 0, v, n, draws, None, dg)
    o_st, _, o_dg = oracle.lcg_draw(M, G, CC, seeds, draws, want_u=False)
    assert np.array_equal(u64(v), o_st)
    assert np.array_equal(u64(dg), o_dg)


@pytest.mark.parametrize("mode", ["hash", "stride"])
def test_draw_host_buffers_match_the_device_call(env, oracle, mode):
    """mc_lcg_draw_host (host buffers, two device slots, a copy stream)
    returns the device call's final states and digests bit for bit over a
    range of several 2^22-stream slices with a ragged end, into page-locked
    tensors and into plain numpy arrays; sampled streams equal the oracle."""
    mc, ctx, torch = env
    n, id0, draws = 2 * 2**22 + 12_345, 77, 64
    spec = (mc.mc_seed_spec(mode=mc.MC_SEED_HASH, seed=W.HASH_SEED) if mode == "hash"
            else mc.mc_seed_spec(mode=mc.MC_SEED_STRIDE, seed=W.STRIDE_X0, stride_q=Q))
    d_st = torch.empty(n, dtype=torch.int64, device="cuda")
    d_dg = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, mc.make_lcg(), spec, id0, d_st, n, draws, None, d_dg)
    ref_st, ref_dg = u64(d_st), u64(d_dg)
    h_st = torch.empty(n, dtype=torch.int64, pin_memory=True)
    h_dg = torch.empty(n, dtype=torch.int64, pin_memory=True)
    mc.mc_lcg_draw_host(ctx, mc.make_lcg(), spec, id0, h_st, n, draws, h_dg)
    assert np.array_equal(h_st.numpy().view(np.uint64), ref_st)
    assert np.array_equal(h_dg.numpy().view(np.uint64), ref_dg)
    a_dg = np.zeros(n, dtype=np.uint64)  # pageable, digests only
    mc.mc_lcg_draw_host(ctx, mc.make_lcg(), spec, id0, None, n, draws, a_dg)
    assert np.array_equal(a_dg, ref_dg)
    idx = np.random.default_rng(5).integers(0, n, 64)
    for i in idx:
        k = id0 + int(i)
        s0 = (oracle.seed_hash(M, W.HASH_SEED, k, 1) if mode == "hash"
              else oracle.seed_stride(M, G, CC, W.STRIDE_X0, Q, k, 1))
        fs, _, dg = oracle.lcg_draw(M, G, CC, s0, draws, want_u=False)
        assert int(fs[0]) == int(ref_st[i]) and int(dg[0]) == int(ref_dg[i])


def test_draw_host_buffers_without_seed_and_errors(env, oracle):
    mc, ctx, torch = env
    n = 2**22 + 5
    st0 = oracle.seed_hash(M, 42, 0, n)
    h_st = st0.copy()
    h_dg = np.zeros(n, dtype=np.uint64)
    mc.mc_lcg_draw_host(ctx, mc.make_lcg(), None, 0, h_st, n, 9, h_dg)
    fs, _, dg = oracle.lcg_draw(M, G, CC, st0[:1000], 9, want_u=False)
    assert np.array_equal(h_st[:1000], fs) and np.array_equal(h_dg[:1000], dg)
    fs, _, dg = oracle.lcg_draw(M, G, CC, st0[-7:], 9, want_u=False)
    assert np.array_equal(h_st[-7:], fs) and np.array_equal(h_dg[-7:], dg)
    with pytest.raises(mc.McError):  # no seed and no states
        mc.mc_lcg_draw_host(ctx, mc.make_lcg(), None, 0, None, 10, 4, h_dg)
    spec = mc.mc_seed_spec(mode=mc.MC_SEED_HASH, seed=42)
    with pytest.raises(mc.McError):  # no output
        mc.mc_lcg_draw_host(ctx, mc.make_lcg(), spec, 0, None, 10, 4, None)

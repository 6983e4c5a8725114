"""Degenerate and edge cases through the C ABI against the oracle: empty
problems (alone and between others in one batched launch), a single
history, no absorption at all (c = 1), LCG widths of 1 and 8 bits, the
smallest pulse problem, and an empty box."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W
from paper_2403_06362_gb300._ffi import MC_NCOUNT

pytestmark = pytest.mark.gpu

G, CC = W.LCG_G, 1


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


def slab_gpu(env, probs):
    mc, ctx, torch = env
    total = sum(p["n_histories"] for p in probs)
    tally = mc.Tally(W.tally_slots(probs), len(probs), n_histories=total)
    cp = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    mc.mc_transport_run(ctx, mc.make_lcg(), cp, mc.mc_run_config(), tally.c)
    torch.cuda.synchronize()
    return tally, cp


def slab_oracle(oracle, probs):
    L = oracle.Lcg(m=63, pad=0, g=G, c=CC)
    size = W.tally_slots(probs)
    tally = np.zeros(size, dtype=np.int64)
    counts, hs = [], []
    for p in probs:
        c = np.zeros(oracle.NCOUNT, dtype=np.uint64)
        r = oracle.slab_run(L, W.to_oracle_problem(p, oracle), tally=tally, counts=c, per_history=True)
        counts.append(c)
        hs.append(r["hist_state"])
    return tally, np.array(counts), np.concatenate(hs)


def test_empty_problem_alone(env):
    mc, ctx, _ = env
    p = [W.slab_problem(10, 1, 0.5, 0, 20, 1, W.SEED_HASH)]
    t, cp = slab_gpu(env, p)
    assert not t.bins.any() and not t.counts.any()
    r = mc.mc_tally_read(ctx, cp, 0, t.c)
    assert r.status == 0 and not r.flux.any()


def test_batched_with_empty_problems_and_a_single_history(env, oracle):
    probs, off = [], 0
    for i, n in enumerate([100, 0, 57, 0, 1, 0]):
        probs.append(W.slab_problem(5 + i, 1.0, 0.7, n, 8, 1, W.SEED_HASH_HIER, tally_offset=off, key=i))
        off += 8
    t, _ = slab_gpu(env, probs)
    tally, counts, hs = slab_oracle(oracle, probs)
    assert np.array_equal(t.bins.cpu().numpy().view(np.int64), tally)
    assert np.array_equal(t.counts.cpu().numpy().view(np.uint64).reshape(-1, MC_NCOUNT)[:, :15], counts[:, :15])
    assert np.array_equal(u64(t.hist_state), hs)


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE])
def test_no_absorption_every_history_leaks(env, oracle, seeding):
    probs = [W.slab_problem(4.0, 1.0, 1.0, 3000, 16, 3, seeding)]
    t, _ = slab_gpu(env, probs)
    tally, counts, hs = slab_oracle(oracle, probs)
    c = t.counts.cpu().numpy().view(np.uint64).reshape(-1, MC_NCOUNT)[0]
    assert c[3] == 0 and c[5] + c[6] == c[0] == 3000  # no absorption; leak low + leak high = sources
    assert np.array_equal(c[:15], counts[0][:15])
    assert np.array_equal(t.bins.cpu().numpy().view(np.int64), tally)
    assert np.array_equal(u64(t.hist_state), hs)


@pytest.mark.parametrize("m", [1, 8])
def test_tiny_widths(env, oracle, m):
    mc, ctx, torch = env
    n, draws = 777, 5
    lcg = mc.make_lcg(m=m, g=G, c=CC)
    v = torch.zeros(n, dtype=torch.int64, device="cuda")
    mc.mc_seed_hash(ctx, lcg, 7, 3, n, v)
    assert np.array_equal(u64(v), oracle.seed_hash(m, 7, 3, n))
    mc.mc_seed_stride(ctx, lcg, 1, 5, 11, n, v)
    seeds = oracle.seed_stride(m, G, CC, 1, 5, 11, n)
    assert np.array_equal(u64(v), seeds)
    u = torch.empty(draws * n, dtype=torch.float64, device="cuda")
    dg = torch.empty(n, dtype=torch.int64, device="cuda")
    mc.mc_lcg_draw(ctx, lcg, None, 0, v, n, draws, u, dg)
    o_st, o_u, o_dg = oracle.lcg_draw(m, G, CC, seeds, draws)
    assert np.array_equal(u64(v), o_st)
    assert np.array_equal(u.cpu().numpy().reshape(draws, n), o_u)
    assert np.array_equal(u64(dg), o_dg)
    assert np.all(o_u < 1.0) and np.all(o_u >= 0.0)


@pytest.mark.parametrize("seeding", [W.SEED_HASH_HIER, W.SEED_STRIDE])
def test_smallest_pulse_problem(env, oracle, seeding):
    mc, ctx, torch = env
    a = W.azurv1(seeding=seeding, n_reps=1, n_batches=1, per_batch=1)
    prob, spec = W.to_mc_pulse(a, mc)
    cp = mc.problem_array([prob])
    t = mc.Tally(W.azurv1_tally_slots(a), 1, n_histories=1)
    mc.mc_transport_run(ctx, mc.make_lcg(), cp, mc.mc_run_config(), t.c)
    torch.cuda.synchronize()
    L = oracle.Lcg(m=63, pad=0, g=G, c=CC)
    o = oracle.azurv1_run(L, W.to_oracle_azurv1(a, oracle), per_history=True)
    assert np.array_equal(t.bins.cpu().numpy().view(np.int64), o["tally"])
    assert np.array_equal(u64(t.hist_state), o["hist_state"])
    del spec


def test_empty_box(env):
    mc, ctx, torch = env
    b = W.box_problem(n_histories=0, seeding=W.SEED_HASH)
    prob, spec = W.to_mc_box(b, mc)
    cp = mc.problem_array([prob])
    t = mc.Tally(W.box_tally_slots(b), 1)
    mc.mc_transport_run(ctx, mc.make_lcg(), cp, mc.mc_run_config(), t.c)
    torch.cuda.synchronize()
    assert not t.bins.any() and not t.counts.any()
    del spec

"""GPU parity of the pulse problem (the paper's Section 5 test) against the
oracle: per-history final states and draw counts bit-exact, counters exact,
collision-estimator tallies within 1e-6 (they are integer multiples of
2^32, so they agree exactly); on a small instance and on sampled histories
of the full 30 x 1000 x 1000 experiment."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W
from paper_2403_06362_gb300._ffi import MC_NCOUNT

pytestmark = pytest.mark.gpu


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


def run_gpu(env, a, hist=True, **cfg):
    mc, ctx, torch = env
    prob, spec = W.to_mc_pulse(a, mc)
    arr = mc.problem_array([prob])
    n = W.azurv1_histories(a)
    tally = mc.Tally(W.azurv1_tally_slots(a), 1, n_histories=n if hist else 0)
    mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(**cfg), tally.c)
    torch.cuda.synchronize()
    tally._keep = (spec, arr)
    return tally


def counts_of(t):
    return t.counts.cpu().numpy().view(np.uint64).reshape(-1, MC_NCOUNT)[0]


def lcg(oracle):
    return oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)


@pytest.mark.parametrize("seeding", [W.SEED_HASH_HIER, W.SEED_HASH, W.SEED_STRIDE])
def test_pulse_parity_small(env, oracle, seeding):
    a = W.azurv1(seeding=seeding, n_reps=2, n_batches=10, per_batch=500)
    t = run_gpu(env, a)
    o = oracle.azurv1_run(lcg(oracle), W.to_oracle_azurv1(a, oracle), per_history=True)
    assert np.array_equal(t.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(t.hist_draws.cpu().numpy().view(np.uint64), o["hist_draws"])
    gc, oc = counts_of(t), o["counts"]
    assert np.array_equal(gc[:15], oc[:15]) and gc[15] == 0
    got = t.bins.cpu().numpy().astype(np.float64)
    exp = o["tally"].astype(np.float64)
    assert np.all(np.abs(got - exp) <= 1e-6 * np.abs(exp))


@pytest.mark.parametrize("seeding", [W.SEED_HASH_HIER, W.SEED_STRIDE])
def test_pulse_full_experiment_sampled(env, oracle, seeding):
    """The paper's experiment at full size (30 x 1000 x 1000 sources) in the
    default launch shape; 300 sampled histories rerun by the oracle."""
    a = W.azurv1(seeding=seeding)
    t = run_gpu(env, a)
    hs = t.hist_state.cpu().numpy().view(np.uint64)
    hd = t.hist_draws.cpu().numpy().view(np.uint64)
    P = W.to_oracle_azurv1(a, oracle)
    rng = np.random.default_rng(3)
    for g in np.unique(rng.integers(0, W.azurv1_histories(a), 300)):
        r = oracle.azurv1_run(lcg(oracle), P, int(g), int(g) + 1, per_history=True)
        assert int(r["hist_state"][0]) == int(hs[g]) and int(r["hist_draws"][0]) == int(hd[g]), g
    c = counts_of(t)
    assert int(c[0]) == W.azurv1_histories(a) and int(c[15]) == 0 and int(c[12]) == 0
    assert int(c[1]) == int(c[2]) + int(c[6])
    assert int(c[2]) == int(c[3]) + int(c[4])
    assert int(c[0]) + int(c[14]) == int(c[3]) + int(c[6])
    assert int(c[7]) == int(c[0]) + int(c[14]) + int(c[1]) + int(c[2]) + 2 * int(c[4])
    # census population per source near exp((k - 1) T) = e^2
    assert abs(int(c[6]) / int(c[0]) - np.exp(2.0)) < 0.05


@pytest.mark.parametrize("block,chunk", [(64, 1), (128, 32), (256, 500)])
def test_pulse_bits_independent_of_launch_shape(env, block, chunk):
    a = W.azurv1(n_reps=1, n_batches=50, per_batch=1000)
    base = run_gpu(env, a, hist=False)
    t = run_gpu(env, a, hist=False, block=block, chunk=chunk)
    assert np.array_equal(base.bins.cpu().numpy(), t.bins.cpu().numpy())
    assert np.array_equal(counts_of(base), counts_of(t))


@pytest.mark.parametrize("seeding,depth", [(W.SEED_HASH_HIER, 1), (W.SEED_HASH, 2), (W.SEED_HASH_HIER, 8)])
def test_pulse_overflow_bank_keeps_the_bits(env, oracle, seeding, depth):
    """Lane stacks of 1, 2 or 8 pending secondaries: the rest wait in the
    device overflow bank and run in later launches; hash-seeded secondaries
    depend only on their seeds (Eq. 5), so every result equals the oracle's
    (whose stack is unbounded)."""
    a = W.azurv1(seeding=seeding, n_reps=2, n_batches=10, per_batch=300)
    t = run_gpu(env, a, stack_depth=depth)
    o = oracle.azurv1_run(lcg(oracle), W.to_oracle_azurv1(a, oracle), per_history=True)
    assert np.array_equal(t.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(t.hist_draws.cpu().numpy().view(np.uint64), o["hist_draws"])
    gc, oc = counts_of(t), o["counts"]
    assert np.array_equal(gc[:15], oc[:15]) and gc[15] == 0
    assert np.array_equal(t.bins.cpu().numpy().view(np.int64), o["tally"])


def test_pulse_stride_stack_overflow_is_reported(env):
    """Stride mode cannot defer a secondary (the family shares one stream in
    depth-first order): a full stack drops it and mc_tally_read reports
    MC_ERR_CAPACITY."""
    mc, ctx, _ = env
    a = W.azurv1(seeding=W.SEED_STRIDE, n_reps=1, n_batches=4, per_batch=200)
    t = run_gpu(env, a, stack_depth=1)
    assert int(counts_of(t)[15]) > 0
    prob, spec = W.to_mc_pulse(a, mc)
    arr = mc.problem_array([prob])
    with pytest.raises(mc.McError):
        mc.mc_tally_read(ctx, arr, 0, t.c)
    del spec


def test_pulse_rejects_bad_stack_depth(env):
    mc, _, _ = env
    a = W.azurv1(n_reps=1, n_batches=2, per_batch=10)
    with pytest.raises(mc.McError):
        run_gpu(env, a, stack_depth=257)


@pytest.mark.parametrize("seeding", [W.SEED_HASH_HIER, W.SEED_STRIDE])
def test_pulse_event_cap_matches_the_oracle_and_is_reported(env, oracle, seeding):
    mc, ctx, _ = env
    a = W.azurv1(seeding=seeding, n_reps=1, n_batches=5, per_batch=200)
    t = run_gpu(env, a, event_cap=4)
    o = oracle.azurv1_run(lcg(oracle), W.to_oracle_azurv1(a, oracle), event_cap=4, per_history=True)
    gc, oc = counts_of(t), o["counts"]
    assert gc[12] > 0 and np.array_equal(gc[:15], oc[:15])
    assert np.array_equal(t.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(t.bins.cpu().numpy().view(np.int64), o["tally"])
    r = mc.mc_tally_read(ctx, t._keep[1], 0, t.c, check=False)
    assert r.status == mc._ffi.MC_ERR_EVENT_CAP

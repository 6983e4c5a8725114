"""GPU parity of the pulse problem in census phases with population control
by one-off hashed values (Section 4; Eq. 5 for the copies) against the
oracle: tallies (integer multiples of the fixed-point unit) and counters
exact, on small instances, over group-aligned id ranges, across launch
shapes (the bank order differs from launch to launch), and on sampled groups
of the full 30 x 1000 x 1000 experiment with 20 phases."""
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


def run_gpu(env, a, tally=None, **cfg):
    mc, ctx, torch = env
    prob, spec = W.to_mc_pulse(a, mc)
    arr = mc.problem_array([prob])
    if tally is None:
        tally = mc.Tally(W.azurv1_tally_slots(a), 1)
    mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(**cfg), tally.c)
    torch.cuda.synchronize()
    tally._keep = (spec, arr)
    return tally


def counts_of(t):
    return t.counts.cpu().numpy().view(np.uint64).reshape(-1, MC_NCOUNT)[0]


def bins_of(t):
    return t.bins.cpu().numpy().view(np.int64)


def lcg(oracle):
    return oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)


def names(oracle, c):
    return dict(zip(oracle.COUNT_NAMES, (int(v) for v in c)))


@pytest.mark.parametrize("seeding,n_census,target", [(W.SEED_HASH_HIER, 8, 0), (W.SEED_HASH, 20, 200),
                                                     (W.SEED_HASH_HIER, 2, 700)])
def test_census_parity_small(env, oracle, seeding, n_census, target):
    a = W.azurv1(seeding=seeding, n_reps=2, n_batches=5, per_batch=300, n_census=n_census, pc_target=target)
    t = run_gpu(env, a)
    o = oracle.azurv1_census_run(lcg(oracle), W.to_oracle_azurv1(a, oracle))
    assert o["status"] == 0
    got, exp = bins_of(t), o["tally"]
    assert np.all(np.abs(got.astype(np.float64) - exp) <= 1e-6 * np.abs(exp.astype(np.float64)))
    assert np.array_equal(got, exp)
    gc, oc = names(oracle, counts_of(t)), names(oracle, o["counts"])
    assert gc == oc
    assert gc["banked"] > 0 and gc["roulette_kills"] + gc["splits"] > 0


def test_census_group_ranges_add_up(env, oracle):
    mc, _, _ = env
    a = W.azurv1(n_reps=1, n_batches=8, per_batch=250, n_census=6)
    whole = run_gpu(env, a)
    t = mc.Tally(W.azurv1_tally_slots(a), 1)
    for lo, hi in [(0, 500), (500, 750), (750, 2000)]:
        run_gpu(env, a, tally=t, range_begin=lo, range_end=hi, accumulate=1)
    assert np.array_equal(bins_of(t), bins_of(whole))
    skip = oracle.COUNT_NAMES.index("max_draws")
    assert np.array_equal(np.delete(counts_of(t), skip), np.delete(counts_of(whole), skip))


@pytest.mark.parametrize("block,chunk", [(64, 1), (256, 64), (128, 128)])
def test_census_bits_independent_of_launch_shape(env, block, chunk):
    # chunks of up to 64 bank items are staged in shared memory, larger ones
    # are read item by item: both give the default launch's bits
    a = W.azurv1(n_reps=1, n_batches=40, per_batch=1000, n_census=10)
    base = run_gpu(env, a)
    t = run_gpu(env, a, block=block, chunk=chunk)
    assert np.array_equal(bins_of(base), bins_of(t))
    assert np.array_equal(counts_of(base), counts_of(t))


def test_census_rejects_stride_and_split_groups(env):
    mc, _, _ = env
    a = W.azurv1(seeding=W.SEED_STRIDE, n_reps=1, n_batches=2, per_batch=10, n_census=4)
    with pytest.raises(mc.McError):
        run_gpu(env, a)
    a = W.azurv1(n_reps=1, n_batches=2, per_batch=10, n_census=4)
    with pytest.raises(mc.McError):
        run_gpu(env, a, range_begin=0, range_end=15)


def test_census_full_experiment_sampled_groups(env, oracle):
    """30 x 1000 x 1000 sources, 20 phases, in the default launch shape;
    the tally rows of 24 sampled (rep, batch) groups rerun by the oracle."""
    a = W.azurv1(n_census=20)
    t = run_gpu(env, a)
    bins = bins_of(t).reshape(-1, a["n_time_bins"])
    c = names(oracle, counts_of(t))
    P = W.to_oracle_azurv1(a, oracle)
    per = a["per_batch"]
    rng = np.random.default_rng(5)
    groups = np.unique(np.concatenate([[0, a["n_reps"] * a["n_batches"] - 1],
                                       rng.integers(0, a["n_reps"] * a["n_batches"], 22)]))
    for g in groups:
        o = oracle.azurv1_census_run(lcg(oracle), P, int(g) * per, (int(g) + 1) * per)
        assert np.array_equal(bins[g], o["tally"].reshape(-1, a["n_time_bins"])[g]), g
    assert c["source"] == W.azurv1_histories(a) and c["dropped"] == 0 and c["capped"] == 0
    assert c["flights"] == c["collisions"] + c["leak_hi"] + c["banked"]
    assert c["source"] + c["children"] + c["splits"] == c["absorptions"] + c["leak_hi"] + c["roulette_kills"]
    # control holds each group near its target: the census at t_end counts
    # about N e^{0.1} per group instead of N e^{2} without control
    assert abs(c["leak_hi"] / W.azurv1_histories(a) - np.exp(0.1)) < 0.01


@pytest.mark.parametrize("depth", [1, 3])
def test_census_overflow_bank_keeps_the_bits(env, oracle, depth):
    a = W.azurv1(n_reps=1, n_batches=6, per_batch=300, n_census=5)
    t = run_gpu(env, a, stack_depth=depth)
    o = oracle.azurv1_census_run(lcg(oracle), W.to_oracle_azurv1(a, oracle))
    assert np.array_equal(bins_of(t), o["tally"])
    assert names(oracle, counts_of(t)) == names(oracle, o["counts"])


def test_census_autotune_uses_whole_groups(env, oracle):
    mc, ctx, torch = env
    a = W.azurv1(n_reps=1, n_batches=7, per_batch=250, n_census=4)
    prob, spec = W.to_mc_pulse(a, mc)
    arr = mc.problem_array([prob])
    t = mc.Tally(W.azurv1_tally_slots(a), 1)
    mc.mc_autotune(ctx, mc.make_lcg(), arr, mc.mc_run_config(), t.c)
    mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(schedule=mc.MC_SCHED_AUTO), t.c)
    torch.cuda.synchronize()
    o = oracle.azurv1_census_run(lcg(oracle), W.to_oracle_azurv1(a, oracle))
    assert np.array_equal(bins_of(t), o["tally"])
    del spec


def test_census_event_cap_matches_the_oracle(env, oracle):
    a = W.azurv1(n_reps=1, n_batches=4, per_batch=200, n_census=4)
    t = run_gpu(env, a, event_cap=2)
    o = oracle.azurv1_census_run(lcg(oracle), W.to_oracle_azurv1(a, oracle), event_cap=2)
    gc, oc = names(oracle, counts_of(t)), names(oracle, o["counts"])
    assert gc["capped"] > 0 and gc == oc
    assert np.array_equal(bins_of(t), o["tally"])

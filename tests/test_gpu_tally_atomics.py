"""Warp-aggregated tally atomics (lanes adding to one slot combine their
values and one lane adds the sum) against one atomic per lane and
contribution: int64 addition is associative, so every kernel must give the
same tally bits, counters and per-history results either way."""
import pytest

from paper_2403_06362_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PER_LANE, AGGREGATED = 1, 2


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


def run(env, kind, spec, n_hist, slots, n_probs, **cfg):
    mc, ctx, torch = env
    keep = None
    if kind == "slab":
        arr = mc.problem_array([W.to_mc_problem(p, mc) for p in spec])
    elif kind == "box":
        prob, keep = W.to_mc_box(spec, mc)
        arr = mc.problem_array([prob])
    else:
        prob, keep = W.to_mc_pulse(spec, mc)
        arr = mc.problem_array([prob])
    tally = mc.Tally(slots, n_probs, n_histories=n_hist)
    mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(**cfg), tally.c)
    torch.cuda.synchronize()
    del keep
    return tally


def assert_same(env, kind, spec, n_hist, slots, n_probs, **cfg):
    torch = env[2]
    a = run(env, kind, spec, n_hist, slots, n_probs, tally_atomics=PER_LANE, **cfg)
    b = run(env, kind, spec, n_hist, slots, n_probs, tally_atomics=AGGREGATED, **cfg)
    assert torch.count_nonzero(a.bins) > 0
    assert torch.equal(a.bins, b.bins)
    assert torch.equal(a.counts, b.counts)
    if n_hist:
        assert torch.equal(a.hist_state, b.hist_state)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("tally_mode", [1, 2])  # staged in shared memory, global atomics
@pytest.mark.parametrize("schedule", [0, 1])
def test_slab(env, precision, tally_mode, schedule):
    if schedule == 1 and tally_mode == 1:
        pytest.skip("the event schedule adds to global memory only")
    probs = W.slab_small(W.SEED_HASH, n_histories=20_000)
    assert_same(env, "slab", probs, 20_000, W.tally_slots(probs), 1, precision=precision,
                tally_mode=tally_mode, schedule=schedule)


def test_slab_batched_and_long(env):
    probs = W.slab_batched(W.SEED_HASH_HIER, n_problems=32, max_histories=4000)
    n = sum(p["n_histories"] for p in probs)
    assert_same(env, "slab", probs, n, W.tally_slots(probs), len(probs))
    probs = W.slab_long(W.SEED_STRIDE, n_histories=5000)
    assert_same(env, "slab", probs, 5000, W.tally_slots(probs), 1)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("schedule", [0, 1])
def test_box(env, precision, schedule):
    b = W.box_problem(n_histories=20_000, seeding=W.SEED_HASH)
    assert_same(env, "box", b, 20_000, W.box_tally_slots(b), 1, precision=precision, schedule=schedule)


@pytest.mark.parametrize("seeding,n_census", [(W.SEED_HASH_HIER, 0), (W.SEED_STRIDE, 0), (W.SEED_HASH_HIER, 5)])
def test_pulse(env, seeding, n_census):
    a = W.azurv1(seeding=seeding, n_reps=2, n_batches=20, per_batch=500, n_census=n_census)
    assert_same(env, "pulse", a, W.azurv1_histories(a), W.azurv1_tally_slots(a), 1)


def test_bad_tally_atomics_rejected(env):
    mc = env[0]
    probs = W.slab_small(W.SEED_HASH, n_histories=100)
    with pytest.raises(mc.McError) as e:
        run(env, "slab", probs, 0, W.tally_slots(probs), 1, tally_atomics=3)
    assert e.value.status == mc._ffi.MC_ERR_ARG

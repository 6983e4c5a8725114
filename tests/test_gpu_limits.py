"""Failure detection on the GPU without a fault: every bounded wait of a run
is driven to its limit through mc_ctx_set_limits (a bound of 0), and the run
must either keep its bits (the slab kernel's compaction-pool lock, whose
give-up path skips the hand-over) or return MC_ERR_TIMEOUT from the host
loop (event schedules, box children, pulse overflow generations), never
hang; the context then runs the same workload correctly with the default
bounds restored."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture()
def env():
    import torch
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import _build
    _build.build()
    ctx = mc.Context(0)
    yield mc, ctx, torch
    torch.cuda.synchronize()
    ctx.close()


def limits(mc, **kw):
    lim = mc.mc_limits(pool_lock_attempts=1 << 20, box_generations=10000, pulse_generations=100000,
                       reserved=0, event_iterations=2**64 - 1)
    for k, v in kw.items():
        setattr(lim, k, v)
    return lim


def slab(mc, ctx, torch, probs, **cfg):
    total = sum(p["n_histories"] for p in probs)
    tally = mc.Tally(W.tally_slots(probs), len(probs), n_histories=total)
    arr = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(**cfg), tally.c)
    torch.cuda.synchronize()
    tally._keep = arr
    return tally


def test_default_limits_read_back(env):
    mc, ctx, _ = env
    got = mc.mc_ctx_get_limits(ctx)
    assert (got.pool_lock_attempts, got.box_generations, got.pulse_generations, got.event_iterations) == \
        (1 << 20, 10000, 100000, 2**64 - 1)
    bad = limits(mc, reserved=1)
    with pytest.raises(mc.McError) as e:
        mc.mc_ctx_set_limits(ctx, bad)
    assert e.value.status == mc._ffi.MC_ERR_ARG


@pytest.mark.parametrize("precision", [0, 1])
def test_pool_lock_that_never_succeeds_keeps_every_bit(env, precision):
    """Long chains thin the warps out, so the default run hands particles
    through the pool; with 0 lock attempts no warp ever takes the lock, every
    warp keeps its own particles, and no particle is counted as dropped."""
    mc, ctx, torch = env
    probs = W.slab_long(W.SEED_HASH, n_histories=20_000)
    ref = slab(mc, ctx, torch, probs, precision=precision, block=256)
    mc.mc_ctx_set_limits(ctx, limits(mc, pool_lock_attempts=0))
    got = slab(mc, ctx, torch, probs, precision=precision, block=256)
    assert torch.equal(got.bins, ref.bins)
    assert torch.equal(got.counts, ref.counts)
    assert torch.equal(got.hist_state, ref.hist_state)
    r = mc.mc_tally_read(ctx, got._keep, 0, got.c)  # raises on MC_ERR_CAPACITY
    assert r.counts["dropped"] == 0
    # the graph-captured launch takes the bound as a kernel argument too
    got_g = slab(mc, ctx, torch, probs, precision=precision, block=256, use_graph=1)
    assert torch.equal(got_g.bins, ref.bins)


@pytest.mark.parametrize("use_graph", [0, 1])
def test_slab_event_schedule_times_out_then_recovers(env, use_graph):
    mc, ctx, torch = env
    # more histories than the tail kernel takes at once, so iterations are needed
    probs = W.slab_small(W.SEED_STRIDE, n_histories=400_000)
    ref = slab(mc, ctx, torch, probs)
    mc.mc_ctx_set_limits(ctx, limits(mc, event_iterations=0))
    with pytest.raises(mc.McError) as e:
        slab(mc, ctx, torch, probs, schedule=1, use_graph=use_graph)
    assert e.value.status == mc._ffi.MC_ERR_TIMEOUT
    # one batch of iterations: here the live particles fall below the tail
    # threshold within it, and the tail kernel finishes the run
    mc.mc_ctx_set_limits(ctx, limits(mc, event_iterations=1))
    got = slab(mc, ctx, torch, probs, schedule=1, use_graph=use_graph)
    assert torch.equal(got.bins, ref.bins)
    mc.mc_ctx_set_limits(ctx, None)
    got = slab(mc, ctx, torch, probs, schedule=1, use_graph=use_graph)
    assert torch.equal(got.bins, ref.bins) and torch.equal(got.hist_state, ref.hist_state)


def box_run(mc, ctx, torch, b, **cfg):
    prob, spec = W.to_mc_box(b, mc)
    arr = mc.problem_array([prob])
    tally = mc.Tally(W.box_tally_slots(b), 1, n_histories=b["n_histories"])
    mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(**cfg), tally.c)
    torch.cuda.synchronize()
    tally._keep = (spec, arr)
    return tally


@pytest.mark.parametrize("schedule", [0, 1])
def test_box_generations_time_out_then_recover(env, schedule):
    mc, ctx, torch = env
    b = W.box_problem(n_histories=3000, seeding=W.SEED_HASH)
    ref = box_run(mc, ctx, torch, b)
    r = mc.mc_tally_read(ctx, ref._keep[1], 0, ref.c)
    assert r.counts["children"] > 0  # the weight windows split: generations follow
    mc.mc_ctx_set_limits(ctx, limits(mc, box_generations=0))
    with pytest.raises(mc.McError) as e:
        box_run(mc, ctx, torch, b, schedule=schedule)
    assert e.value.status == mc._ffi.MC_ERR_TIMEOUT
    if schedule == 1:
        # more sources than the tail kernel takes at once: iterations are needed
        big = W.box_problem(n_histories=200_000, seeding=W.SEED_HASH)
        mc.mc_ctx_set_limits(ctx, limits(mc, event_iterations=0))
        with pytest.raises(mc.McError) as e:
            box_run(mc, ctx, torch, big, schedule=schedule)
        assert e.value.status == mc._ffi.MC_ERR_TIMEOUT
    mc.mc_ctx_set_limits(ctx, None)
    got = box_run(mc, ctx, torch, b, schedule=schedule)
    assert torch.equal(got.bins, ref.bins) and torch.equal(got.hist_state, ref.hist_state)


@pytest.mark.parametrize("n_census", [0, 4])
def test_pulse_overflow_generations_time_out_then_recover(env, n_census):
    """A one-entry lane stack sends secondaries to the overflow bank, which
    the host follows generation by generation; with a bound of 0 the first
    generation already times out."""
    mc, ctx, torch = env
    a = W.azurv1(seeding=W.SEED_HASH_HIER, n_reps=1, n_batches=4, per_batch=200, n_census=n_census)

    def run(**cfg):
        prob, spec = W.to_mc_pulse(a, mc)
        arr = mc.problem_array([prob])
        tally = mc.Tally(W.azurv1_tally_slots(a), 1, n_histories=W.azurv1_histories(a))
        mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(**cfg), tally.c)
        torch.cuda.synchronize()
        tally._keep = (spec, arr)
        return tally

    ref = run(stack_depth=1)
    mc.mc_ctx_set_limits(ctx, limits(mc, pulse_generations=0))
    with pytest.raises(mc.McError) as e:
        run(stack_depth=1)
    assert e.value.status == mc._ffi.MC_ERR_TIMEOUT
    mc.mc_ctx_set_limits(ctx, None)
    got = run(stack_depth=1)
    assert torch.equal(got.bins, ref.bins) and torch.equal(got.counts, ref.counts)
    assert np.array_equal(got.hist_state.cpu().numpy(), ref.hist_state.cpu().numpy())

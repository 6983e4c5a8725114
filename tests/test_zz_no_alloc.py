"""mc_transport_run_static, the entry point for callers that cannot allocate
device memory (code whose device memory belongs to another allocator, or
that must not grow its footprint after start-up; it needs no mc_ctx and keeps
its scratch in a fixed device array inside libmc), must give the same
results as mc_transport_run, call after call, even though every call reuses
the array the previous call left behind.  Both entry points make the same
int64 tally contributions, so the bins must be equal bit for bit (within the
1e-6 relative bar of the other parity tests, which equality meets).  This
file is collected last so that a run stopping at the first failure has run
every other test first."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-6


def run_both(mc, ctx, torch, probs):
    lcg = mc.make_lcg()
    total = sum(p["n_histories"] for p in probs)
    arr = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    cfg = mc.mc_run_config()
    ref = mc.Tally(W.tally_slots(probs), len(probs), n_histories=total)
    mc.mc_transport_run(ctx, lcg, arr, cfg, ref.c)
    got = mc.Tally(W.tally_slots(probs), len(probs), n_histories=total)
    mc.mc_transport_run_static(lcg, arr, cfg, got.c)
    torch.cuda.synchronize()
    return ref, got


def test_static_entry_matches_context_entry_on_consecutive_calls():
    import torch
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import _build
    _build.build()
    ctx = mc.Context(0)
    # two different calls in a row: the second sees what the first left in
    # the shared array (more problems, a nonzero ticket)
    for probs in (W.slab_batched(W.SEED_HASH_HIER, n_problems=40, max_histories=5000),
                  W.slab_small(W.SEED_STRIDE)):
        ref, got = run_both(mc, ctx, torch, probs)
        rb = ref.bins.cpu().numpy().astype(np.float64)
        gb = got.bins.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(gb - rb) <= TOL * np.abs(rb))
        assert torch.equal(got.bins, ref.bins)
        assert torch.equal(got.counts, ref.counts)
        assert torch.equal(got.hist_state, ref.hist_state)
        assert torch.equal(got.hist_draws, ref.hist_draws)
    ctx.close()


def test_static_entry_matches_the_oracle(oracle):
    """The static entry against the oracle directly: final state and draw
    count of every history bit-exact, counters exact, int64 bins within the
    1e-6 relative bar, for several problems in one call."""
    import torch
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import _build
    _build.build()
    probs = W.slab_batched(W.SEED_HASH_HIER, n_problems=12, max_histories=3000)
    total = sum(p["n_histories"] for p in probs)
    arr = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    got = mc.Tally(W.tally_slots(probs), len(probs), n_histories=total)
    mc.mc_transport_run_static(mc.make_lcg(), arr, mc.mc_run_config(), got.c)
    torch.cuda.synchronize()
    tally = np.zeros(W.tally_slots(probs), dtype=np.int64)
    hs, hd, counts = [], [], []
    for p in probs:
        c = np.zeros(oracle.NCOUNT, dtype=np.uint64)
        r = oracle.slab_run(oracle.Lcg(m=W.LCG_M, pad=0, g=W.LCG_G, c=W.LCG_C),
                            W.to_oracle_problem(p, oracle), tally=tally, counts=c, per_history=True)
        hs.append(r["hist_state"])
        hd.append(r["hist_draws"])
        counts.append(c)
    assert np.array_equal(got.hist_state.cpu().numpy().view(np.uint64),
                          np.concatenate(hs).astype(np.uint64))
    assert np.array_equal(got.hist_draws.cpu().numpy().view(np.uint64),
                          np.concatenate(hd).astype(np.uint64))
    gc = got.counts.cpu().numpy().view(np.uint64).reshape(len(probs), -1)
    assert np.array_equal(gc[:, :14], np.array(counts)[:, :14])
    gb = got.bins.cpu().numpy().astype(np.float64)
    ob = tally.astype(np.float64)
    assert np.all(np.abs(gb - ob) <= TOL * np.abs(ob))


def test_static_entry_rejects_too_many_problems():
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import _build
    _build.build()
    probs = W.slab_batched(W.SEED_HASH_HIER, n_problems=257, max_histories=10)
    tally = mc.Tally(W.tally_slots(probs), len(probs))
    arr = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    with pytest.raises(mc.McError) as e:
        mc.mc_transport_run_static(mc.make_lcg(), arr, mc.mc_run_config(), tally.c)
    assert e.value.status == mc._ffi.MC_ERR_ARG and "256" in str(e.value)


def test_static_entry_at_its_problem_maximum():
    """256 problems, the largest call the fixed array holds, after a call
    with fewer problems."""
    import torch
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import _build
    _build.build()
    ctx = mc.Context(0)
    for n in (3, 256):
        probs = W.slab_batched(W.SEED_STRIDE, n_problems=n, max_histories=400)
        ref, got = run_both(mc, ctx, torch, probs)
        assert torch.equal(got.bins, ref.bins)
        assert torch.equal(got.counts, ref.counts)
        assert torch.equal(got.hist_state, ref.hist_state)
    ctx.close()


def test_static_entry_rejects_other_geometries():
    import paper_2403_06362_gb300 as mc
    from paper_2403_06362_gb300 import _build
    _build.build()
    b = W.box_problem(n_histories=10)
    prob, spec = W.to_mc_box(b, mc)
    tally = mc.Tally(W.box_tally_slots(b), 1)
    with pytest.raises(mc.McError) as e:
        mc.mc_transport_run_static(mc.make_lcg(), mc.problem_array([prob]), mc.mc_run_config(), tally.c)
    assert e.value.status == mc._ffi.MC_ERR_ARG and "not a slab problem" in str(e.value)
    del spec

"""GPU parity of the slab transport (mc_transport_run / mc_tally_read)
against the oracle: per-history final RNG state and draw count bit-exact,
integer counters exact, int64 tallies within 1e-6 relative (fp64 path), and
tally bits identical across launch shapes, staging modes and id ranges."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W
from paper_2403_06362_gb300._ffi import MC_NCOUNT

pytestmark = pytest.mark.gpu

M, G, CC, Q = W.LCG_M, W.LCG_G, W.LCG_C, W.STRIDE_Q
TOL = 1e-6


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


def olcg(oracle):
    return oracle.Lcg(m=M, pad=0, g=G, c=CC)


def gpu_run(env, probs, n_hist_out=True, **cfg_kw):
    mc, ctx, torch = env
    total = sum(p["n_histories"] for p in probs)
    tally = mc.Tally(W.tally_slots(probs), len(probs), n_histories=total if n_hist_out else 0)
    cprobs = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    cfg = mc.mc_run_config(**cfg_kw)
    mc.mc_transport_run(ctx, mc.make_lcg(), cprobs, cfg, tally.c)
    torch.cuda.synchronize()
    return tally, cprobs


def oracle_run(oracle, probs, per_history=True):
    size = W.tally_slots(probs)
    tally = np.zeros(size, dtype=np.int64)
    tf = np.zeros(size)
    counts, hs, hd = [], [], []
    for p in probs:
        c = np.zeros(oracle.NCOUNT, dtype=np.uint64)
        r = oracle.slab_run(olcg(oracle), W.to_oracle_problem(p, oracle), tally=tally, tally_fp=tf,
                            counts=c, per_history=per_history)
        counts.append(c)
        if per_history:
            hs.append(r["hist_state"])
            hd.append(r["hist_draws"])
    out = dict(tally=tally, tally_fp=tf, counts=np.array(counts))
    if per_history:
        out["hist_state"] = np.concatenate(hs)
        out["hist_draws"] = np.concatenate(hd)
    return out


def assert_tally_close(got, exp):
    got = np.asarray(got, dtype=np.int64)
    exp = np.asarray(exp, dtype=np.int64)
    diff = np.abs(got.astype(np.float64) - exp.astype(np.float64))
    assert np.all(diff <= TOL * np.abs(exp.astype(np.float64))), (np.max(diff), np.argmax(diff))


def counts_of(tally, n):
    return tally.counts.cpu().numpy().view(np.uint64).reshape(n, MC_NCOUNT)


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE, W.SEED_HASH_HIER])
def test_slab_small_parity(env, oracle, seeding):
    probs = W.slab_small(seeding)
    tally, cprobs = gpu_run(env, probs)
    o = oracle_run(oracle, probs)
    assert np.array_equal(tally.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(tally.hist_draws.cpu().numpy().view(np.uint64), o["hist_draws"])
    assert np.array_equal(counts_of(tally, 1)[:, :14], o["counts"][:, :14])
    assert_tally_close(tally.bins.cpu().numpy(), o["tally"])
    mc = env[0]
    r = mc.mc_tally_read(env[1], cprobs, 0, tally.c)
    h = probs[0]["L"] / probs[0]["n_bins"]
    exp_flux = o["tally"].reshape(10, 20).sum(0) * 2.0**-32 / (probs[0]["n_histories"] * h)
    assert np.allclose(r.flux, exp_flux, rtol=1e-6, atol=0)
    assert r.counts["source"] == probs[0]["n_histories"]


@pytest.mark.parametrize("block,chunk,mode", [(64, 1, 1), (128, 7, 2), (256, 128, 0), (512, 4096, 1),
                                              (32, 32, 2)])
def test_tally_bits_independent_of_launch_shape(env, oracle, block, chunk, mode):
    probs = W.slab_small(W.SEED_HASH, n_histories=20_000)
    base, _ = gpu_run(env, probs, n_hist_out=False)
    t, _ = gpu_run(env, probs, n_hist_out=False, block=block, chunk=chunk, tally_mode=mode)
    assert np.array_equal(t.bins.cpu().numpy(), base.bins.cpu().numpy())
    assert np.array_equal(counts_of(t, 1), counts_of(base, 1))


@pytest.mark.parametrize("precision", [0, 1])
def test_large_blocks_with_staged_tally_and_pool(env, precision):
    """512-thread blocks with a 4000-slot shared-memory tally, the edge
    tables and the compaction pool: over 48 KiB of shared memory with the
    kernel's static part; the bits equal the default launch's."""
    probs = W.slab_long(W.SEED_HASH, n_histories=20_000)
    base, _ = gpu_run(env, probs, n_hist_out=False, precision=precision)
    for block in (512, 128):
        t, _ = gpu_run(env, probs, n_hist_out=False, precision=precision, block=block)
        assert np.array_equal(t.bins.cpu().numpy(), base.bins.cpu().numpy())
        assert np.array_equal(counts_of(t, 1), counts_of(base, 1))


def test_staged_tally_near_the_shared_memory_limit(env, oracle):
    """A 25 600-slot tally forced into shared memory (200 KiB): with the edge
    tables and the compaction pool it would not fit, so the launch gives them
    up; the bits equal the global-atomic run's and the oracle's."""
    probs = [W.slab_problem(50.0, 1.0, 0.9, 4000, 2560, 10, W.SEED_HASH)]
    staged, _ = gpu_run(env, probs, tally_mode=1)
    direct, _ = gpu_run(env, probs, n_hist_out=False, tally_mode=2)
    assert np.array_equal(staged.bins.cpu().numpy(), direct.bins.cpu().numpy())
    assert np.array_equal(counts_of(staged, 1), counts_of(direct, 1))
    o = oracle_run(oracle, probs)
    assert np.array_equal(staged.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert_tally_close(staged.bins.cpu().numpy(), o["tally"])


def test_ranges_accumulate_to_the_same_bits(env):
    mc, ctx, torch = env
    probs = W.slab_small(W.SEED_STRIDE, n_histories=20_000)
    base, cprobs = gpu_run(env, probs, n_hist_out=False)
    tally = mc.Tally(W.tally_slots(probs), 1)
    for i, (a, b) in enumerate([(0, 1), (1, 7001), (7001, 19999), (19999, 20000)]):
        cfg = mc.mc_run_config(range_begin=a, range_end=b, accumulate=1 if i else 0)
        mc.mc_transport_run(ctx, mc.make_lcg(), cprobs, cfg, tally.c)
    torch.cuda.synchronize()
    assert np.array_equal(tally.bins.cpu().numpy(), base.bins.cpu().numpy())
    c1, c0 = counts_of(tally, 1), counts_of(base, 1)
    assert np.array_equal(c1[:, :13], c0[:, :13])


@pytest.mark.parametrize("precision", [0, 1])
def test_bin_tables_in_global_memory(env, oracle, precision):
    """Bin edge and width tables read from global memory: one problem with
    more bins than the shared-memory table holds, and a batched launch with
    uneven bin counts; fp64 tallies against the oracle, and batched tallies
    (fp64 and fp32-guarded) bit for bit against each problem run alone."""
    one = [W.slab_problem(60.0, 1.0, 0.9, 4000, 6000, 2, W.SEED_HASH)]
    t, _ = gpu_run(env, one, precision=precision)
    c = counts_of(t, 1)[0]
    assert int(c[0]) == 4000 == int(c[3]) + int(c[5]) + int(c[6])
    if precision == 0:
        o = oracle_run(oracle, one)
        assert np.array_equal(t.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
        assert_tally_close(t.bins.cpu().numpy(), o["tally"])
    probs, off = [], 0
    for i, (L, nb) in enumerate([(7.0, 3), (30.0, 700), (2.5, 1), (45.0, 5000), (12.0, 64)]):
        probs.append(W.slab_problem(L, 1.0, 0.8, 1500, nb, 2, W.SEED_HASH_HIER, tally_offset=off, key=i))
        off += 2 * nb
    t, _ = gpu_run(env, probs, precision=precision)
    if precision == 0:
        o = oracle_run(oracle, probs)
        assert np.array_equal(t.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
        assert_tally_close(t.bins.cpu().numpy(), o["tally"])
    bins = t.bins.cpu().numpy()
    for p in probs:
        alone = dict(p, tally_offset=0)
        a, _ = gpu_run(env, [alone], n_hist_out=False, precision=precision)
        lo, n = p["tally_offset"], 2 * p["n_bins"]
        assert np.array_equal(a.bins.cpu().numpy()[:n], bins[lo:lo + n])


def test_pure_absorber_beam_closed_form_on_gpu(env):
    mc, ctx, torch = env
    S, L, nb = 1.0, 4.0, 8
    p = W.slab_problem(L, S, 0.0, 1_000_000, nb, 20, W.SEED_HASH, source=W.SRC_BEAM)
    tally, cprobs = gpu_run(env, [p], n_hist_out=False)
    r = mc.mc_tally_read(ctx, cprobs, 0, tally.c)
    e = np.linspace(0, L, nb + 1)
    exact = (np.exp(-S * e[:-1]) - np.exp(-S * e[1:])) / (S * (e[1:] - e[:-1]))
    assert np.all(np.abs(r.flux - exact) < 4.5 * r.rel_err * r.flux)


def test_batched_problems_parity(env, oracle):
    # uneven problems in one launch; histories capped so the oracle is quick
    probs = W.slab_batched(W.SEED_HASH_HIER, n_problems=24, max_histories=3000)
    tally, _ = gpu_run(env, probs)
    o = oracle_run(oracle, probs)
    assert np.array_equal(tally.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(counts_of(tally, len(probs))[:, :14], o["counts"][:, :14])
    assert_tally_close(tally.bins.cpu().numpy(), o["tally"])
    probs = W.slab_batched(W.SEED_STRIDE, n_problems=24, max_histories=3000)
    tally, _ = gpu_run(env, probs)
    o = oracle_run(oracle, probs)
    assert np.array_equal(tally.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert_tally_close(tally.bins.cpu().numpy(), o["tally"])


def test_long_chains_full_size_sampled(env, oracle):
    """10^6 histories of the 200 cm, c = 0.9999 slab (stride seeding), in the
    default launch shape; 400 sampled histories rerun one by one in the
    oracle must match in final state and draw count, and the stride
    exceedance counters must agree with the per-history draw counts."""
    probs = W.slab_long(W.SEED_STRIDE)
    tally, _ = gpu_run(env, probs)
    hs = tally.hist_state.cpu().numpy().view(np.uint64)
    hd = tally.hist_draws.cpu().numpy().view(np.uint64)
    rng = np.random.default_rng(1)
    sample = np.unique(rng.integers(0, probs[0]["n_histories"], 400))
    P = W.to_oracle_problem(probs[0], oracle)
    for i in sample:
        r = oracle.slab_run(olcg(oracle), P, int(i), int(i) + 1, per_history=True)
        assert int(r["hist_state"][0]) == int(hs[i]) and int(r["hist_draws"][0]) == int(hd[i]), i
    c = counts_of(tally, 1)[0]
    d = hd.astype(np.int64)
    assert int(c[8]) == int(np.sum(d > Q))
    assert int(c[9]) == int(np.sum(np.maximum(d - Q, 0)))
    assert int(c[7]) == int(d.sum()) and int(c[13]) == int(d.max())
    assert int(c[0]) == int(c[3]) + int(c[5]) + int(c[6])


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE])
def test_long_chains_tally_parity_on_every_batch(env, oracle, seeding):
    """The full long-chain slab (L = 200, c = 0.9999, 200 bins, 20 batches of
    5·10^4 ids): the first 1000 ids of every batch, run through
    range_begin/range_end into one tally (20 accumulating calls), against
    the oracle on the same ids.  Every one of the 20 x 200 slots within 1e-6
    relative, counters exact, per-history final states and draw counts
    exact.  The GPU's flight logarithm and the oracle's differ by one ulp on
    about 0.2 % of inputs; a leak/collide decision flipped by that would show
    as a history whose final state differs, and is reported by id."""
    mc, ctx, torch = env
    probs = W.slab_long(seeding)
    p = probs[0]
    n, nbat, nb, per = p["n_histories"], p["n_batches"], p["n_bins"], 1000
    tally = mc.Tally(W.tally_slots(probs), 1, n_histories=n)
    cprobs = mc.problem_array([W.to_mc_problem(q, mc) for q in probs])
    starts = [b * n // nbat for b in range(nbat)]
    assert all((s0 * nbat) // n == b and ((s0 + per - 1) * nbat) // n == b for b, s0 in enumerate(starts))
    for b, s0 in enumerate(starts):
        cfg = mc.mc_run_config(range_begin=s0, range_end=s0 + per, accumulate=1 if b else 0)
        mc.mc_transport_run(ctx, mc.make_lcg(), cprobs, cfg, tally.c)
    torch.cuda.synchronize()
    P = W.to_oracle_problem(p, oracle)
    size = W.tally_slots(probs)
    ot = np.zeros(size, dtype=np.int64)
    oc = np.zeros(oracle.NCOUNT, dtype=np.uint64)
    hs = tally.hist_state.cpu().numpy().view(np.uint64)
    hd = tally.hist_draws.cpu().numpy().view(np.uint64)
    flips = []
    for s0 in starts:
        r = oracle.slab_run(olcg(oracle), P, s0, s0 + per, tally=ot, counts=oc, per_history=True)
        bad = np.nonzero((hs[s0:s0 + per] != r["hist_state"]) | (hd[s0:s0 + per] != r["hist_draws"]))[0]
        flips += [s0 + int(i) for i in bad]
    assert not flips, f"histories whose final state or draw count differ: {flips[:20]}"
    got = tally.bins.cpu().numpy().reshape(nbat, nb)
    exp = ot.reshape(nbat, nb)
    assert np.count_nonzero(exp) == nbat * nb  # every slot scored: the comparison covers all 4000
    assert_tally_close(got, exp)
    gc = counts_of(tally, 1)[0]
    assert np.array_equal(gc[:13], oc[:13]) and gc[13] == oc[13], (gc, oc)
    assert int(gc[0]) == nbat * per


def test_event_cap_reported(env):
    mc, ctx, torch = env
    p = W.slab_problem(200.0, 1.0, 0.9999, 500, 10, 1, W.SEED_HASH)
    tally, cprobs = gpu_run(env, [p], n_hist_out=False, event_cap=50)
    r = mc.mc_tally_read(ctx, cprobs, 0, tally.c, check=False)
    assert r.status == mc._ffi.MC_ERR_EVENT_CAP and r.counts["capped"] > 0


def test_fp32_guarded_error_stated(env, oracle):
    # fp32 flight against the fp64 oracle on the same histories: the fp32
    # path carries its position as a pair of floats and re-decides near a
    # face in fp64, so its histories follow the fp64 ones; per-bin tallies
    # agree to about 1e-7 relative (bound 1e-5 here).
    probs = W.slab_small(W.SEED_HASH, n_histories=200_000)
    probs[0]["n_batches"] = 20
    t32, _ = gpu_run(env, probs, precision=1)
    o = oracle_run(oracle, probs)
    g = t32.bins.cpu().numpy().reshape(20, 20).sum(0).astype(np.float64)
    e = o["tally"].reshape(20, 20).sum(0).astype(np.float64)
    rel = np.abs(g - e) / e
    assert rel.max() < 1e-5, rel.max()
    diverged = int(np.count_nonzero(t32.hist_state.cpu().numpy().view(np.uint64) != o["hist_state"]))
    assert diverged <= 2, diverged
    c32 = counts_of(t32, 1)[0]
    assert int(c32[0]) == int(c32[3]) + int(c32[5]) + int(c32[6])


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE])
def test_fp32_guarded_long_chains_follow_fp64(env, seeding):
    """10^4 collisions per history: the fp32 path's position pairs keep its
    histories on the fp64 trajectories (no decision flipped in 3·10^4
    histories, about 1.4·10^8 flights), and every bin agrees within 1e-5
    relative."""
    probs = W.slab_long(seeding, n_histories=30_000)
    t64, _ = gpu_run(env, probs, precision=0)
    t32, _ = gpu_run(env, probs, precision=1)
    diverged = int((t64.hist_state != t32.hist_state).sum().item())
    assert diverged <= 3, diverged
    a = t64.bins.cpu().numpy().astype(np.float64)
    b = t32.bins.cpu().numpy().astype(np.float64)
    nz = a != 0
    assert np.max(np.abs(a[nz] - b[nz]) / a[nz]) < 1e-5


def _same_bits(a, b, n):
    assert np.array_equal(a.bins.cpu().numpy(), b.bins.cpu().numpy())
    assert np.array_equal(counts_of(a, n), counts_of(b, n))
    if a.hist_state is not None and b.hist_state is not None:
        assert np.array_equal(a.hist_state.cpu().numpy(), b.hist_state.cpu().numpy())
        assert np.array_equal(a.hist_draws.cpu().numpy(), b.hist_draws.cpu().numpy())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("which", ["small_hash", "small_stride", "batched", "long"])
def test_event_schedule_bit_identical_to_history(env, oracle, precision, use_graph, which):
    if which == "small_hash":
        probs = W.slab_small(W.SEED_HASH)
    elif which == "small_stride":
        probs = W.slab_small(W.SEED_STRIDE)
    elif which == "batched":
        probs = W.slab_batched(W.SEED_HASH_HIER, n_problems=30, max_histories=4000)
    else:
        probs = W.slab_long(W.SEED_STRIDE, n_histories=5000)
    hist, _ = gpu_run(env, probs, precision=precision)
    ev, _ = gpu_run(env, probs, precision=precision, schedule=1, use_graph=use_graph)
    _same_bits(hist, ev, len(probs))
    if precision == 0 and which == "small_hash":
        o = oracle_run(oracle, probs)
        assert np.array_equal(ev.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
        assert_tally_close(ev.bins.cpu().numpy(), o["tally"])


@pytest.mark.parametrize("precision", [0, 1])
def test_event_schedule_refills_a_full_bank(env, precision):
    """More histories than the bank's 2^21 slots: ended slots take new
    histories from the ticket inside the iteration kernel for many
    iterations before the tail kernel; the bits equal the history
    schedule's."""
    probs = W.slab_small(W.SEED_STRIDE, n_histories=3_000_000)
    hist, _ = gpu_run(env, probs, precision=precision)
    for use_graph in (0, 1):
        ev, _ = gpu_run(env, probs, precision=precision, schedule=1, use_graph=use_graph)
        _same_bits(hist, ev, 1)


def test_event_schedule_event_cap_and_ranges(env):
    mc, ctx, torch = env
    p = [W.slab_problem(200.0, 1.0, 0.9999, 300, 10, 1, W.SEED_HASH)]
    a, _ = gpu_run(env, p, event_cap=40)
    b, _ = gpu_run(env, p, event_cap=40, schedule=1)
    _same_bits(a, b, 1)
    assert counts_of(b, 1)[0, 12] > 0
    # a sub-range in event mode equals the same sub-range in history mode
    probs = W.slab_small(W.SEED_HASH)
    a, _ = gpu_run(env, probs, range_begin=123, range_end=4567)
    b, _ = gpu_run(env, probs, range_begin=123, range_end=4567, schedule=1)
    _same_bits(a, b, 1)


def test_autotune_leaves_tally_alone_and_auto_matches(env):
    mc, ctx, torch = env
    probs = W.slab_batched(W.SEED_HASH_HIER, n_problems=40, max_histories=20_000)
    cprobs = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    tally = mc.Tally(W.tally_slots(probs), len(probs))
    tally.bins.fill_(12345)
    best, ms = mc.mc_autotune(ctx, mc.make_lcg(), cprobs, mc.mc_run_config(), tally.c)
    torch.cuda.synchronize()
    assert int(tally.bins.min()) == 12345 and int(tally.bins.max()) == 12345
    # block 0 with chunk 0: the library's default shape, which the full-range
    # check keeps when no sampled shape beats it on the whole range
    assert ms > 0 and best.schedule in (0, 1) and best.block in (0, 128, 256, 512)
    assert (best.block == 0) == (best.chunk == 0)
    ref, _ = gpu_run(env, probs, n_hist_out=False)
    auto, _ = gpu_run(env, probs, n_hist_out=False, schedule=2)
    again, _ = gpu_run(env, probs, n_hist_out=False, schedule=2)
    _same_bits(ref, auto, len(probs))
    _same_bits(ref, again, len(probs))


def test_history_graph_replay_with_new_problem_data(env):
    mc, ctx, torch = env
    a = W.slab_batched(W.SEED_HASH_HIER, n_problems=16, max_histories=5000, seed=7)
    b = W.slab_batched(W.SEED_HASH_HIER, n_problems=16, max_histories=5000, seed=8)
    # same shape (count, totals differ -> force equal totals by capping all)
    for p in a + b:
        p["n_histories"] = 5000
    tally = mc.Tally(W.tally_slots(a), len(a), n_histories=16 * 5000)
    for probs in (a, b, a):
        cp = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
        mc.mc_transport_run(ctx, mc.make_lcg(), cp, mc.mc_run_config(use_graph=1), tally.c)
        torch.cuda.synchronize()
        ref, _ = gpu_run(env, probs)
        _same_bits(ref, tally, len(probs))


def test_history_graph_with_other_history_counts(env):
    """The same problem shapes with other history counts: the history range
    is baked into a captured launch, so each count gets its own graph."""
    mc, ctx, torch = env
    tally = None  # one tally for every call: the same buffers, so only the counts differ
    for n in (3000, 7000, 3000, 12000):
        probs = W.slab_batched(W.SEED_HASH_HIER, n_problems=8, max_histories=n, seed=5)
        for p in probs:
            p["n_histories"] = n
        if tally is None:
            tally = mc.Tally(W.tally_slots(probs), len(probs))
        cp = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
        mc.mc_transport_run(ctx, mc.make_lcg(), cp, mc.mc_run_config(use_graph=1), tally.c)
        torch.cuda.synchronize()
        ref, _ = gpu_run(env, probs, n_hist_out=False)
        _same_bits(ref, tally, len(probs))


def test_tally_overflow_reported(env):
    mc, ctx, torch = env
    probs = W.slab_small(W.SEED_HASH, n_histories=100)
    tally, cprobs = gpu_run(env, probs, n_hist_out=False)
    tally.bins[7] = 2**62  # a bin at the headroom limit
    r = mc.mc_tally_read(ctx, cprobs, 0, tally.c, check=False)
    assert r.status == mc._ffi.MC_ERR_OVERFLOW


def test_batched_full_size_sampled(env, oracle):
    """All 256 batched problems at full size (~4e7 histories, one launch,
    fp64, default shape); 300 sampled histories rerun by the oracle."""
    probs = W.slab_batched(W.SEED_HASH_HIER)
    tally, _ = gpu_run(env, probs)
    hs = tally.hist_state.cpu().numpy().view(np.uint64)
    hd = tally.hist_draws.cpu().numpy().view(np.uint64)
    starts = np.cumsum([0] + [p["n_histories"] for p in probs])
    rng = np.random.default_rng(11)
    for g in np.unique(rng.integers(0, starts[-1], 300)):
        k = int(np.searchsorted(starts, g, side="right") - 1)
        P = W.to_oracle_problem(probs[k], oracle)
        i = int(g - starts[k])
        r = oracle.slab_run(olcg(oracle), P, i, i + 1, per_history=True)
        assert int(r["hist_state"][0]) == int(hs[g]) and int(r["hist_draws"][0]) == int(hd[g]), g
    c = counts_of(tally, len(probs))
    assert np.array_equal(c[:, 0], np.array([p["n_histories"] for p in probs], dtype=np.uint64))
    assert np.array_equal(c[:, 0], c[:, 3] + c[:, 5] + c[:, 6])


# The cooperative tail: a launch of a few long-chain histories in blocks of
# 256 threads ends with every block's last warp holding at most four live
# histories, which it runs with lane groups (draw-only values ahead, one lane
# for the chain of positions, the group for the tallies).  Blocks of 32
# threads have no pool and never take that path, so the two launch shapes
# must give the same bits; and the oracle fixes both, event caps included
# (a cap then falls inside a round of the tail).
def long_few(seeding, n):
    return W.slab_long(seeding, n_histories=n)


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE])
@pytest.mark.parametrize("cap", [0, 2500])
def test_cooperative_tail_matches_oracle(env, oracle, seeding, cap):
    probs = long_few(seeding, 96)
    tally, _ = gpu_run(env, probs, block=256, event_cap=cap)
    size = W.tally_slots(probs)
    t = np.zeros(size, dtype=np.int64)
    c = np.zeros(oracle.NCOUNT, dtype=np.uint64)
    o = oracle.slab_run(olcg(oracle), W.to_oracle_problem(probs[0], oracle), tally=t, counts=c,
                        per_history=True, event_cap=cap if cap else 2**40)
    assert np.array_equal(tally.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(tally.hist_draws.cpu().numpy().view(np.uint64), o["hist_draws"])
    assert np.array_equal(counts_of(tally, 1)[0, :14], c[:14])
    if cap:
        assert c[12] > 0  # some histories were capped (MC_C_CAPPED)
    assert_tally_close(tally.bins.cpu().numpy(), t)


@pytest.mark.parametrize("precision", [0, 1])
def test_cooperative_tail_same_bits_as_one_lane_path(env, precision):
    probs = long_few(W.SEED_HASH, 200)
    coop, _ = gpu_run(env, probs, block=256, precision=precision)
    plain, _ = gpu_run(env, probs, block=32, precision=precision)
    import torch
    assert torch.equal(coop.bins, plain.bins)
    assert torch.equal(coop.counts, plain.counts)
    assert torch.equal(coop.hist_state, plain.hist_state)
    assert torch.equal(coop.hist_draws, plain.hist_draws)


@pytest.mark.parametrize("m", [62, 48])
@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE])
def test_other_modulus_with_cooperative_tail(env, oracle, m, seeding):
    """Another modulus runs the kernels' generic-modulus instantiation, the
    cooperative tail's included (few long histories, blocks of 256)."""
    mc, ctx, torch = env
    probs = long_few(seeding, 64)
    tally = mc.Tally(W.tally_slots(probs), 1, n_histories=64)
    cprobs = mc.problem_array([W.to_mc_problem(p, mc) for p in probs])
    mc.mc_transport_run(ctx, mc.make_lcg(m=m, g=G, c=CC), cprobs, mc.mc_run_config(block=256), tally.c)
    torch.cuda.synchronize()
    t = np.zeros(W.tally_slots(probs), dtype=np.int64)
    c = np.zeros(oracle.NCOUNT, dtype=np.uint64)
    o = oracle.slab_run(oracle.Lcg(m=m, pad=0, g=G, c=CC), W.to_oracle_problem(probs[0], oracle), tally=t,
                        counts=c, per_history=True)
    assert np.array_equal(tally.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(tally.hist_draws.cpu().numpy().view(np.uint64), o["hist_draws"])
    assert np.array_equal(counts_of(tally, 1)[0, :14], c[:14])
    assert_tally_close(tally.bins.cpu().numpy(), t)

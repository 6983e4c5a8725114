"""GPU parity of the two-region box transport against the oracle (primary
final states and draw counts bit-exact, counters exact, the 64^3 mesh tally
within 1e-6 relative), and bit-identity of the event-based schedule with the
history-based one -- the property Eq. (5)'s on-demand child seeds provide."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W
from paper_2403_06362_gb300._ffi import MC_NCOUNT

pytestmark = pytest.mark.gpu

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


def gpu_box(env, b, hist=True, **cfg):
    mc, ctx, torch = env
    prob, spec = W.to_mc_box(b, mc)
    arr = mc.problem_array([prob])
    tally = mc.Tally(W.box_tally_slots(b), 1, n_histories=b["n_histories"] if hist else 0)
    mc.mc_transport_run(ctx, mc.make_lcg(), arr, mc.mc_run_config(**cfg), tally.c)
    torch.cuda.synchronize()
    tally._keep = (spec, arr)
    return tally


def counts_of(t):
    return t.counts.cpu().numpy().view(np.uint64).reshape(-1, MC_NCOUNT)[0]


def oracle_box(oracle, b):
    L = oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)
    return oracle.box_run(L, W.to_oracle_box(b, oracle), per_history=True)


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE, W.SEED_HASH_HIER])
def test_box_parity_with_oracle(env, oracle, seeding):
    b = W.box_problem(n_histories=4000, seeding=seeding)
    t = gpu_box(env, b)
    o = oracle_box(oracle, b)
    assert np.array_equal(t.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(t.hist_draws.cpu().numpy().view(np.uint64), o["hist_draws"])
    oc = o["counts"]
    gc = counts_of(t)
    assert np.array_equal(gc[:13], oc[:13]) and gc[13] == oc[13] and gc[14] == oc[14]
    assert gc[10] > 0 and gc[11] > 0  # splits and roulette both happened
    got = t.bins.cpu().numpy().astype(np.float64)
    exp = o["tally"].astype(np.float64)
    assert np.all(np.abs(got - exp) <= TOL * np.abs(exp))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_box_event_schedule_bit_identical(env, precision, use_graph):
    b = W.box_problem(n_histories=20_000)
    h = gpu_box(env, b, precision=precision)
    e = gpu_box(env, b, precision=precision, schedule=1, use_graph=use_graph)
    assert np.array_equal(h.bins.cpu().numpy(), e.bins.cpu().numpy())
    assert np.array_equal(counts_of(h), counts_of(e))
    assert np.array_equal(h.hist_state.cpu().numpy(), e.hist_state.cpu().numpy())


@pytest.mark.parametrize("precision", [0, 1])
def test_box_event_schedule_refills_a_full_bank(env, precision):
    """More source histories than the bank's 2^21 slots, so ended slots take
    new histories (and, in later generations, split children) from the
    ticket inside the iteration kernel; bits equal the history schedule's."""
    b = W.box_problem(n_histories=2_500_000, seeding=W.SEED_STRIDE)
    h = gpu_box(env, b, precision=precision)
    e = gpu_box(env, b, precision=precision, schedule=1, use_graph=1)
    assert np.array_equal(h.bins.cpu().numpy(), e.bins.cpu().numpy())
    assert np.array_equal(counts_of(h), counts_of(e))
    assert np.array_equal(h.hist_state.cpu().numpy(), e.hist_state.cpu().numpy())
    assert np.array_equal(h.hist_draws.cpu().numpy(), e.hist_draws.cpu().numpy())


@pytest.mark.parametrize("block,chunk", [(64, 1), (128, 32), (512, 256)])
def test_box_bits_independent_of_launch_shape(env, block, chunk):
    b = W.box_problem(n_histories=20_000, seeding=W.SEED_STRIDE)
    base = gpu_box(env, b, hist=False)
    t = gpu_box(env, b, hist=False, block=block, chunk=chunk)
    assert np.array_equal(base.bins.cpu().numpy(), t.bins.cpu().numpy())
    assert np.array_equal(counts_of(base), counts_of(t))


def test_box_ranges_accumulate(env):
    mc, ctx, torch = env
    b = W.box_problem(n_histories=6000)
    base = gpu_box(env, b, hist=False)
    prob, spec = W.to_mc_box(b, mc)
    arr = mc.problem_array([prob])
    tally = mc.Tally(W.box_tally_slots(b), 1)
    for i, (lo, hi) in enumerate([(0, 1000), (1000, 1001), (1001, 6000)]):
        mc.mc_transport_run(ctx, mc.make_lcg(), arr,
                            mc.mc_run_config(range_begin=lo, range_end=hi, accumulate=1 if i else 0), tally.c)
    torch.cuda.synchronize()
    assert np.array_equal(tally.bins.cpu().numpy(), base.bins.cpu().numpy())


def test_box_fp32_error_stated(env, oracle):
    b = W.box_problem(n_histories=20_000)
    t32 = gpu_box(env, b, hist=False, precision=1)
    o = oracle_box(oracle, b)
    g = t32.bins.cpu().numpy().astype(np.float64).sum()
    e = o["tally"].astype(np.float64).sum()
    assert abs(g - e) / e < 2e-2
    c = counts_of(t32)
    assert int(c[0]) + int(c[14]) == int(c[6]) + int(c[11]) + int(c[12])


def test_box_auto_schedule_matches(env):
    b = W.box_problem(n_histories=30_000)
    ref = gpu_box(env, b, hist=False)
    auto = gpu_box(env, b, hist=False, schedule=2)
    assert np.array_equal(ref.bins.cpu().numpy(), auto.bins.cpu().numpy())
    assert np.array_equal(counts_of(ref), counts_of(auto))


def test_box_full_size_sampled(env, oracle):
    """10^8 source histories (the benchmark's box) in the default launch
    shape, fp64; 200 sampled histories rerun one by one by the oracle must
    match in the primary's final state and draw count."""
    b = W.box_large(W.SEED_HASH)
    t = gpu_box(env, b)
    hs = t.hist_state.cpu().numpy().view(np.uint64)
    hd = t.hist_draws.cpu().numpy().view(np.uint64)
    L = oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)
    P = W.to_oracle_box(b, oracle)
    rng = np.random.default_rng(5)
    for i in np.unique(rng.integers(0, b["n_histories"], 200)):
        r = oracle.box_run(L, P, int(i), int(i) + 1, per_history=True)
        assert int(r["hist_state"][0]) == int(hs[i]) and int(r["hist_draws"][0]) == int(hd[i]), i
    c = counts_of(t)
    assert int(c[0]) == b["n_histories"] and int(c[12]) == 0
    assert int(c[0]) + int(c[14]) == int(c[6]) + int(c[11])


def test_box_event_cap_matches_the_oracle_and_is_reported(env, oracle):
    """A per-particle flight cap of 3: the capped particles, draws and tallies
    equal the oracle's under the same cap, and mc_tally_read reports
    MC_ERR_EVENT_CAP."""
    mc, ctx, _ = env
    b = W.box_problem(n_histories=3000, seeding=W.SEED_HASH)
    t = gpu_box(env, b, event_cap=3)
    L = oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)
    o = oracle.box_run(L, W.to_oracle_box(b, oracle), event_cap=3, per_history=True)
    gc, oc = counts_of(t), o["counts"]
    assert gc[12] > 0 and np.array_equal(gc[:15], oc[:15])
    assert np.array_equal(t.hist_state.cpu().numpy().view(np.uint64), o["hist_state"])
    assert np.array_equal(t.bins.cpu().numpy().view(np.int64), o["tally"])
    r = mc.mc_tally_read(ctx, t._keep[1], 0, t.c, check=False)
    assert r.status == mc._ffi.MC_ERR_EVENT_CAP

"""Pins of the oracle's slab transport against closed forms of one-speed
transport theory, exact balance identities and the stride bookkeeping of
Section 3 (exceedance of a stride; Section 1 cites its tally bias).

Closed forms used (per source particle, track-length flux averaged over bin
[a, b] of a slab [0, L] with total cross section S):
  pure absorber, beam at x = 0, mu = 1:
      (exp(-S a) - exp(-S b)) / (S (b - a))
  pure absorber, isotropic source uniform in [0, L]:
      [2 - (E3(S a) - E3(S b) + E3(S (L-b)) - E3(S (L-a))) / (S (b - a))] / (2 S L)
"""
import numpy as np
import pytest
from scipy.special import expn

from paper_2403_06362_gb300 import workloads as W

LCG = dict(m=63, g=2806196910506780709, c=1)


def lcg(oracle):
    return oracle.Lcg(m=LCG["m"], pad=0, g=LCG["g"], c=LCG["c"])


def run(oracle, p, **kw):
    return oracle.slab_run(lcg(oracle), W.to_oracle_problem(p, oracle), **kw)


def batch_flux(res, p):
    nb, nbat, N = p["n_bins"], p["n_batches"], p["n_histories"]
    h = p["L"] / nb
    t = res["tally"][p["tally_offset"]:p["tally_offset"] + nb * nbat].reshape(nbat, nb)
    per = N // nbat
    return t.astype(np.float64) * 2.0**-32 / (per * h)


def check_against(phi_b, exact, z=4.5):
    mean = phi_b.mean(axis=0)
    se = phi_b.std(axis=0, ddof=1) / np.sqrt(phi_b.shape[0])
    dev = np.abs(mean - exact) / se
    assert np.all(dev < z), (dev, mean, exact)
    return dev


def test_beam_pure_absorber_closed_form(oracle):
    S, L, nb = 1.0, 4.0, 8
    p = W.slab_problem(L, S, 0.0, 200_000, nb, 20, W.SEED_HASH, source=W.SRC_BEAM)
    res = run(oracle, p)
    e = np.linspace(0, L, nb + 1)
    exact = (np.exp(-S * e[:-1]) - np.exp(-S * e[1:])) / (S * (e[1:] - e[:-1]))
    check_against(batch_flux(res, p), exact)


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE])
def test_isotropic_pure_absorber_closed_form(oracle, seeding):
    S, L, nb = 1.3, 5.0, 10
    p = W.slab_problem(L, S, 0.0, 200_000, nb, 20, seeding)
    res = run(oracle, p)
    e = np.linspace(0, L, nb + 1)
    a, b = e[:-1], e[1:]
    e3 = lambda x: expn(3, x)  # noqa: E731
    exact = (2.0 - (e3(S * a) - e3(S * b) + e3(S * (L - b)) - e3(S * (L - a))) / (S * (b - a))) / (2 * S * L)
    check_against(batch_flux(res, p), exact)


@pytest.mark.parametrize("seeding", [W.SEED_HASH, W.SEED_STRIDE, W.SEED_HASH_HIER])
def test_balance_identities(oracle, seeding):
    p = W.slab_small(seeding)[0]
    c = dict(zip(oracle.COUNT_NAMES, (int(v) for v in run(oracle, p)["counts"])))
    assert c["source"] == p["n_histories"]
    assert c["source"] == c["absorptions"] + c["leak_lo"] + c["leak_hi"]
    assert c["flights"] == c["collisions"] + c["leak_lo"] + c["leak_hi"]
    assert c["collisions"] == c["absorptions"] + c["scatters"]
    # isotropic source: 2 draws; then one per flight, per collision, per scatter
    assert c["draws"] == 2 * c["source"] + c["flights"] + c["collisions"] + c["scatters"]
    assert c["capped"] == 0 and c["exceed_hist"] == 0


def test_infinite_medium_collisions(oracle):
    # Far from the faces every history collides 1/(1 - c) times on average.
    c_ratio = 0.9
    p = W.slab_problem(1.0e4, 1.0, c_ratio, 20_000, 1, 1, W.SEED_HASH)
    cnt = dict(zip(oracle.COUNT_NAMES, (int(v) for v in run(oracle, p)["counts"])))
    mean = cnt["collisions"] / cnt["source"]
    se = np.sqrt(c_ratio / (1 - c_ratio) ** 2 / cnt["source"])
    assert abs(mean - 1.0 / (1.0 - c_ratio)) < 4.5 * se


def test_collision_rate_equals_sigma_t_times_track(oracle):
    # E[collisions] = Sigma_t E[track length] in any medium.
    S = 1.7
    p = W.slab_problem(6.0, S, 0.7, 100_000, 12, 20, W.SEED_HASH)
    res = run(oracle, p)
    cnt = dict(zip(oracle.COUNT_NAMES, (int(v) for v in res["counts"])))
    track = res["tally_fp"].sum()
    # sd of collisions per history < 1/(1-c) scale; loose 5-sigma bound
    se = np.sqrt((0.7 / 0.3**2 + 1.0) / cnt["source"]) * cnt["source"]
    assert abs(cnt["collisions"] - S * track) < 5 * se


def test_fixed_point_close_to_fp64_shadow(oracle):
    p = W.slab_small(W.SEED_HASH)[0]
    res = run(oracle, p)
    fixed = res["tally"].astype(np.float64) * 2.0**-32
    flights = int(res["counts"][1])
    # each contribution rounds by at most 2^-33; a flight touches <= 3 bins here
    assert np.all(np.abs(fixed - res["tally_fp"]) <= 3 * flights * 2.0**-33)
    assert np.allclose(fixed, res["tally_fp"], rtol=1e-9, atol=0)


def test_ranges_add_up_exactly(oracle):
    # int64 tallies are associative: any split of the histories sums to the
    # same bits, which is what makes schedules and launch shapes irrelevant.
    p = W.slab_small(W.SEED_HASH)[0]
    L = lcg(oracle)
    P = W.to_oracle_problem(p, oracle)
    whole = oracle.slab_run(L, P)
    t = np.zeros_like(whole["tally"])
    tf = np.zeros_like(whole["tally_fp"])
    cnt = np.zeros_like(whole["counts"])
    for a, b in [(0, 17), (17, 5000), (5000, 9999), (9999, 10000)]:
        oracle.slab_run(L, P, a, b, tally=t, tally_fp=tf, counts=cnt)
    assert np.array_equal(t, whole["tally"])
    assert np.array_equal(cnt[:13], whole["counts"][:13])


def test_batches_hold_their_own_histories(oracle):
    p = W.slab_small(W.SEED_HASH)[0]
    L = lcg(oracle)
    P = W.to_oracle_problem(p, oracle)
    whole = oracle.slab_run(L, P)["tally"].reshape(10, 20)
    for k in (0, 3, 9):
        part = oracle.slab_run(L, P, k * 1000, (k + 1) * 1000)["tally"].reshape(10, 20)
        assert np.array_equal(part[k], whole[k])
        assert not np.any(np.delete(part, k, axis=0))


def test_stride_exceedance_bookkeeping(oracle):
    # Per-history draw counts against a deliberately short stride Q.
    q = 9
    p = W.slab_problem(10.0, 1.0, 0.8, 3000, 20, 10, W.SEED_STRIDE, stride_q=q)
    res = run(oracle, p, per_history=True)
    d = res["hist_draws"].astype(np.int64)
    cnt = dict(zip(oracle.COUNT_NAMES, (int(v) for v in res["counts"])))
    assert cnt["exceed_hist"] == int(np.sum(d > q)) > 0
    assert cnt["exceed_draws"] == int(np.sum(np.maximum(d - q, 0)))
    assert cnt["max_draws"] == int(d.max())
    assert cnt["draws"] == int(d.sum())


def test_stride_overlap_when_stride_exceeded(oracle):
    # With stride Q, history k+1 starts exactly where history k would be after
    # Q draws: a history that draws more than Q reuses its successor's numbers.
    q = 9
    p = W.slab_problem(10.0, 1.0, 0.8, 50, 20, 1, W.SEED_STRIDE, stride_q=q)
    L = lcg(oracle)
    P = W.to_oracle_problem(p, oracle)
    for k in range(10):
        sk = oracle.slab_seed(L, P, k)
        assert oracle.lcg_skip(sk, q, 63, LCG["g"], LCG["c"]) == oracle.slab_seed(L, P, k + 1)


def test_final_state_is_seed_advanced_by_draws(oracle):
    p = W.slab_small(W.SEED_HASH, n_histories=500)[0]
    L = lcg(oracle)
    P = W.to_oracle_problem(p, oracle)
    res = oracle.slab_run(L, P, per_history=True)
    for i in range(0, 500, 37):
        s = oracle.slab_seed(L, P, i)
        assert s == oracle.hash_seed(i, 42, 63)
        assert oracle.lcg_skip(s, int(res["hist_draws"][i]), 63, LCG["g"], LCG["c"]) == int(res["hist_state"][i])


def test_event_cap(oracle):
    p = W.slab_problem(200.0, 1.0, 0.9999, 200, 10, 1, W.SEED_HASH)
    res = run(oracle, p, event_cap=50)
    cnt = dict(zip(oracle.COUNT_NAMES, (int(v) for v in res["counts"])))
    assert res["status"] == 1 and cnt["capped"] > 0
    assert cnt["flights"] <= 50 * 200


def test_hash_and_stride_agree_statistically(oracle):
    out = {}
    for s in (W.SEED_HASH, W.SEED_STRIDE):
        p = W.slab_problem(10.0, 1.0, 0.5, 100_000, 20, 20, s)
        out[s] = batch_flux(run(oracle, p), p)
    m0, m1 = out[0].mean(0), out[1].mean(0)
    se = np.sqrt(out[0].var(0, ddof=1) / 20 + out[1].var(0, ddof=1) / 20)
    assert np.all(np.abs(m0 - m1) < 5 * se)

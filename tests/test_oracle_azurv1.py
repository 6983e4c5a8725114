"""Pins of the oracle's supercritical time-dependent problem (Section 5's
AZURV1-like test) against branching-process closed forms.  With collision
rate Sigma_t v = 1 and k = c nu = 1.1 secondaries per collision on average,
the expected population is N(t) = exp((k - 1) t), so per source particle:
  particles alive at census T:         exp((k - 1) T)
  collisions in [a, b):                (exp((k - 1) b) - exp((k - 1) a)) / (k - 1)
and every particle ends by absorption or census (exact balance)."""
import numpy as np
import pytest

from paper_2403_06362_gb300 import workloads as W

K = 0.4 * 2.75


def lcg(oracle):
    return oracle.Lcg(m=63, pad=0, g=W.LCG_G, c=1)


def counts(oracle, r):
    return dict(zip(oracle.COUNT_NAMES, (int(v) for v in r["counts"])))


def chunked(oracle, a, chunks):
    """Per-chunk counts and tallies, for batch standard errors."""
    P = W.to_oracle_azurv1(a, oracle)
    total = W.azurv1_histories(a)
    per = total // chunks
    cs, ts = [], []
    for i in range(chunks):
        r = oracle.azurv1_run(lcg(oracle), P, i * per, (i + 1) * per)
        cs.append(counts(oracle, r))
        ts.append(r["tally"].reshape(-1, a["n_time_bins"]).sum(axis=0))
    return cs, np.array(ts, dtype=np.float64), per


@pytest.mark.parametrize("seeding", [W.SEED_HASH_HIER, W.SEED_STRIDE])
def test_census_population_and_collisions(oracle, seeding):
    a = W.azurv1(seeding=seeding, n_reps=1, n_batches=40, per_batch=1000)
    cs, _, per = chunked(oracle, a, 40)
    census = np.array([c["leak_hi"] / per for c in cs])
    coll = np.array([c["collisions"] / per for c in cs])
    se = lambda v: v.std(ddof=1) / np.sqrt(len(v))  # noqa: E731
    assert abs(census.mean() - np.exp((K - 1) * 20)) < 4.5 * se(census)
    assert abs(coll.mean() - (np.exp((K - 1) * 20) - 1) / (K - 1)) < 4.5 * se(coll)


def test_time_bins_match_population_growth(oracle):
    # count every collision (x_half huge): bin j expects
    # (exp(0.1 (j+1)) - exp(0.1 j)) / 0.1 per source
    a = W.azurv1(n_reps=1, n_batches=40, per_batch=1000, x_half=1e300)
    _, ts, per = chunked(oracle, a, 40)
    per_src = ts * 2.0**-32 / per
    j = np.arange(20)
    exp = (np.exp((K - 1) * (j + 1)) - np.exp((K - 1) * j)) / (K - 1)
    se = per_src.std(axis=0, ddof=1) / np.sqrt(per_src.shape[0])
    assert np.all(np.abs(per_src.mean(axis=0) - exp) < 4.5 * se)


@pytest.mark.parametrize("seeding", [W.SEED_HASH_HIER, W.SEED_STRIDE, W.SEED_HASH])
def test_exact_balances(oracle, seeding):
    a = W.azurv1(seeding=seeding, n_reps=2, n_batches=5, per_batch=500)
    c = counts(oracle, oracle.azurv1_run(lcg(oracle), W.to_oracle_azurv1(a, oracle)))
    assert c["source"] == 5000
    assert c["flights"] == c["collisions"] + c["leak_hi"]
    assert c["collisions"] == c["absorptions"] + c["scatters"]
    assert c["source"] + c["children"] == c["absorptions"] + c["leak_hi"] + c["capped"]
    # draws: a direction per particle, one per flight, one per collision, one
    # multiplicity and one new direction per scattering
    assert c["draws"] == (c["source"] + c["children"]) + c["flights"] + c["collisions"] + 2 * c["scatters"]
    # multiplicity floor(2.75 + u): 1 or 2 secondaries, mean 1.75
    assert c["scatters"] <= c["children"] <= 2 * c["scatters"]


def test_multiplicity_mean(oracle):
    a = W.azurv1(n_reps=1, n_batches=20, per_batch=1000)
    c = counts(oracle, oracle.azurv1_run(lcg(oracle), W.to_oracle_azurv1(a, oracle)))
    frac = (c["children"] - c["scatters"]) / c["scatters"]  # fraction with 3 outgoing
    assert abs(frac - 0.75) < 4.5 * np.sqrt(0.75 * 0.25 / c["scatters"])


def test_seeds_follow_eq4_and_stride(oracle):
    L = lcg(oracle)
    a = W.azurv1(n_reps=3, n_batches=4, per_batch=5)
    P = W.to_oracle_azurv1(a, oracle)
    g = (2 * 4 + 3) * 5 + 1  # rep 2, batch 3, particle 1
    assert oracle.azurv1_seed(L, P, g) == oracle.hash_seed(1, oracle.hash64(3, oracle.hash64(2, 42)), 63)
    s = W.azurv1(seeding=W.SEED_STRIDE, n_reps=3, n_batches=4, per_batch=5)
    assert oracle.azurv1_seed(L, W.to_oracle_azurv1(s, oracle), g) == oracle.stride_seed(1, W.STRIDE_Q, g, 63,
                                                                                          W.LCG_G, 1)


def test_ranges_add_up(oracle):
    L = lcg(oracle)
    for seeding in (W.SEED_HASH_HIER, W.SEED_STRIDE):
        a = W.azurv1(seeding=seeding, n_reps=1, n_batches=4, per_batch=500)
        P = W.to_oracle_azurv1(a, oracle)
        whole = oracle.azurv1_run(L, P)
        t = np.zeros_like(whole["tally"])
        c = np.zeros_like(whole["counts"])
        for lo, hi in [(0, 700), (700, 701), (701, 2000)]:
            oracle.azurv1_run(L, P, lo, hi, tally=t, counts=c)
        assert np.array_equal(t, whole["tally"])
        assert np.array_equal(c[:13], whole["counts"][:13])

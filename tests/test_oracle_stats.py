"""Pins of the oracle's Section 5 statistics: the Shapiro-Wilk W and p-value
(Royston's AS R94 approximation) against scipy.stats.shapiro, which
implements the same published algorithm, and the normal quantile against
textbook values."""
import numpy as np
import pytest
import scipy.stats as ss


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8, 11, 12, 13, 20, 50, 100, 1000, 5000])
@pytest.mark.parametrize("dist", ["normal", "uniform", "exponential"])
def test_shapiro_wilk_matches_scipy(oracle, n, dist):
    rng = np.random.default_rng(n * 7 + len(dist))
    x = getattr(rng, dist)(size=n)
    w, p = oracle.shapiro_wilk(x)
    ref = ss.shapiro(x)
    assert w == pytest.approx(float(ref.statistic), abs=1e-9)
    assert p == pytest.approx(float(ref.pvalue), rel=1e-6, abs=1e-12)


def test_shapiro_wilk_rejects_bad_input(oracle):
    with pytest.raises(ValueError):
        oracle.shapiro_wilk(np.ones(10))
    with pytest.raises(ValueError):
        oracle.shapiro_wilk(np.arange(2.0))


def test_norm_ppf_textbook_values(oracle):
    assert oracle.norm_ppf(0.5) == pytest.approx(0.0, abs=1e-15)
    assert oracle.norm_ppf(0.975) == pytest.approx(1.959963984540054, abs=1e-13)
    assert oracle.norm_ppf(0.8413447460685429) == pytest.approx(1.0, abs=1e-13)
    for p in (1e-6, 0.01, 0.3, 0.99):
        assert oracle.norm_cdf(oracle.norm_ppf(p)) == pytest.approx(p, rel=1e-12)


def test_pvalues_uniform_under_normality(oracle):
    rng = np.random.default_rng(99)
    ps = [oracle.shapiro_wilk(rng.normal(size=20))[1] for _ in range(400)]
    assert ss.kstest(ps, "uniform").pvalue > 1e-3


def test_batch_stats(oracle):
    rng = np.random.default_rng(5)
    x = rng.normal(loc=3.0, scale=2.0, size=(30, 7))
    z, w, p = oracle.batch_stats(x)
    assert np.allclose(z.mean(axis=0), 0.0, atol=1e-12)
    assert np.allclose(z.std(axis=0, ddof=1), 1.0, atol=1e-12)
    for j in range(7):
        wj, pj = oracle.shapiro_wilk(x[:, j])
        assert w[j] == wj and p[j] == pj

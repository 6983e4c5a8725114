"""Pins of the oracle's LCG (Eq. 1), skip-ahead (Eq. 2), stride seeds
(Section 3) and uniform conversion, against facts the mathematics fixes:
the Hull-Dobell full period, the geometric-series closed form of k steps,
composition of skips, the no-overlap condition QN <= 2^m, and exactness of
the 53-bit uniform."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _params():
    d = {}
    with open(os.path.join(HERE, "golden", "lcg_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                d[k] = int(v)
    return d


P = _params()
M, G, CC, Q = P["m"], P["g"], P["c"], P["Q"]


def closed_form_skip(x0, k, m, g, c):
    """X_k = g^k x0 + c (g^k - 1)/(g - 1) mod 2^m, evaluated exactly with
    integers: (g^k - 1) is reduced mod (g - 1) 2^m, which keeps it divisible
    by (g - 1) and the quotient correct mod 2^m."""
    mod = 1 << m
    big = (g - 1) * mod
    gk_big = pow(g, k, big)
    series = ((gk_big - 1) % big) // (g - 1)
    return (pow(g, k, mod) * x0 + c * series) % mod


def test_parameters_satisfy_hull_dobell():
    # Full period 2^m for c odd and g = 1 mod 4 (Section 2's "chosen correctly").
    assert CC % 2 == 1 and G % 4 == 1


@pytest.mark.parametrize("m", [8, 12, 16])
def test_full_period_by_stepping(oracle, m):
    x = 12345 % (1 << m)
    seen = np.zeros(1 << m, dtype=bool)
    for _ in range(1 << m):
        assert not seen[x]
        seen[x] = True
        x = oracle.lcg_next(x, m, G, CC)
    assert seen.all() and x == 12345 % (1 << m)


@pytest.mark.parametrize("m", [20, 22])
def test_full_period_by_skip(oracle, m):
    # X_0..X_{2^m - 1} by skip-ahead (unit stride) is a permutation of [0, 2^m).
    xs = oracle.seed_stride(m, G, CC, 0, 1, 0, 1 << m)
    assert np.array_equal(np.sort(xs), np.arange(1 << m, dtype=np.uint64))
    assert oracle.lcg_next(int(xs[-1]), m, G, CC) == 0


@pytest.mark.parametrize("g,c", [(G, 2), (G + 2, 1)])
def test_broken_parameters_lose_full_period(oracle, g, c):
    # c even, or g = 3 mod 4, violates Hull-Dobell: the orbit of 0 is short.
    m = 12
    x, n = 0, 0
    while True:
        x = oracle.lcg_next(x, m, g, c)
        n += 1
        if x == 0 or n > (1 << m):
            break
    assert n < (1 << m)


def test_skip_matches_stepping(oracle):
    rng = np.random.default_rng(1)
    for x0 in [1, int(rng.integers(0, 2**63))]:
        x = x0
        for k in range(1, 3001):
            x = oracle.lcg_next(x, M, G, CC)
            if k in (1, 2, 5, 64, 1000, 3000):
                assert oracle.lcg_skip(x0, k, M, G, CC) == x


def test_skip_matches_stepping_one_stride(oracle):
    x = 1
    for _ in range(Q):
        x = oracle.lcg_next(x, M, G, CC)
    assert oracle.lcg_skip(1, Q, M, G, CC) == x


@pytest.mark.parametrize("k", [0, 1, 7, Q, 2 * Q, Q * 2**26, 2**63 - 1, 2**64 - 1])
def test_skip_closed_form(oracle, k):
    for x0 in (1, 0x5DEECE66D, 2**63 - 1):
        assert oracle.lcg_skip(x0, k, M, G, CC) == closed_form_skip(x0, k, M, G, CC)


def test_skip_composition(oracle):
    rng = np.random.default_rng(2)
    for _ in range(50):
        a, b = (int(v) for v in rng.integers(0, 2**40, size=2))
        x0 = int(rng.integers(0, 2**63))
        assert oracle.lcg_skip(oracle.lcg_skip(x0, a, M, G, CC), b, M, G, CC) == \
            oracle.lcg_skip(x0, a + b, M, G, CC)


def test_stride_seed_uses_exact_step_count(oracle):
    # unit k gets X_{Qk} from X_0; Q*k beyond 2^64 is kept exact (128-bit).
    for k in (0, 1, 2, 3, 2**26 - 1, 2**50 + 3):
        assert oracle.stride_seed(1, Q, k, M, G, CC) == closed_form_skip(1, Q * k, M, G, CC)
    assert oracle.stride_seed(1, Q, 0, M, G, CC) == 1
    # consecutive units are exactly Q steps apart
    s = oracle.seed_stride(M, G, CC, 1, Q, 10, 5)
    for a, b in zip(s[:-1], s[1:]):
        assert oracle.lcg_skip(int(a), Q, M, G, CC) == int(b)


def test_stride_no_overlap_iff_qn_fits(oracle):
    # Section 3: N units of stride Q repeat no state iff Q N <= 2^m.
    m, q = 14, 100
    for n, expect_unique in ((163, True), (164, False)):  # 163*100 <= 16384 < 164*100
        seeds = oracle.seed_stride(m, G, CC, 0, q, 0, n)
        states = []
        for s in seeds:
            x = int(s)
            for _ in range(q):
                states.append(x)
                x = oracle.lcg_next(x, m, G, CC)
        assert (len(set(states)) == len(states)) == expect_unique


def test_u01_exact_top_53_bits(oracle):
    rng = np.random.default_rng(3)
    xs = [0, 1, 1023, 1024, 2**62, 2**63 - 1] + [int(v) for v in rng.integers(0, 2**63, size=200)]
    for x in xs:
        u = oracle.u01(x, 63)
        assert 0.0 <= u < 1.0
        assert u * 2.0**53 == float(x >> 10) and (x >> 10) < 2**53
    assert oracle.u01(2**63 - 1, 63) == 1.0 - 2.0**-53
    for x in (0, 5, 2**64 - 1):
        assert oracle.u01(x, 64) * 2.0**53 == float(x >> 11)
    for x in (0, 3, 2**20 - 1):
        assert oracle.u01(x, 20) == x / 2.0**20


def test_draw_digest_and_layout(oracle):
    # draw j of stream i is the uniform of its (j+1)-th state; the digest is
    # the wrapping sum of the draws' IEEE bit patterns.
    seeds = np.array([1, 42, 2**62 + 7], dtype=np.uint64)
    st, u, dg = oracle.lcg_draw(M, G, CC, seeds, 5)
    for i, s in enumerate(seeds):
        x = int(s)
        tot = 0
        for j in range(5):
            x = oracle.lcg_next(x, M, G, CC)
            assert u[j, i] == oracle.u01(x, M)
            tot = (tot + int(np.float64(u[j, i]).view(np.uint64))) % 2**64
        assert int(st[i]) == x and int(dg[i]) == tot

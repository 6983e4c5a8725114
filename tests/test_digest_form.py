"""Host-side checks of the arithmetic the digest kernel (csrc/rng.cu,
draw_digest_m63_kernel) is built on, against the oracle's per-draw digest
(the sum over a stream's draws of the fp64 bit patterns of u, Eq. 1 and the
53-bit uniform).  Everything here is restated in Python integers and numpy
float32; nothing is taken from the CUDA sources.

The kernel's form, for m = 63:
- it steps the doubled state z = 2x mod 2^64 by z' = g z + 2c;
- the uniform's 53 bits are n = z >> 11;
- s is the normalising shift of n, i.e. clz(z >> 32) when z >> 32 != 0;
- the digest is sum(n << s) + (1021 D - sum s) 2^52 mod 2^64 for D draws;
- sum s is kept as the bit pattern of an fp32 subnormal sum, and an
  all-ones s (a zero high word) turns that sum into a NaN."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
M64 = (1 << 64) - 1


def _params():
    d = {}
    with open(os.path.join(HERE, "golden", "lcg_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                d[k] = int(v)
    return d


P = _params()
M, G, CC = P["m"], P["g"], P["c"]
MASK = (1 << M) - 1


def clz32(v):
    return 32 if v == 0 else 32 - v.bit_length()


def summed_digest(x0, draws):
    """(final state, digest, marked) of one stream in the kernel's form;
    marked streams are the ones the kernel redoes per draw."""
    z = (x0 << 1) & M64
    acc, s_sum, marked = 0, 0, False
    for _ in range(draws):
        z = (G * z + 2 * CC) & M64
        zh = z >> 32
        if zh == 0:
            marked = True
            continue
        s = clz32(zh)
        n = z >> 11
        y = n << s
        assert (1 << 52) <= y < (1 << 53)  # leading 1 at bit 52
        acc += y
        s_sum += s
    d = (acc + (((1021 * draws - s_sum) % (1 << 12)) << 52)) & M64
    return z >> 1, d, marked


def start_before(x, k=1):
    """The masked state whose k-th successor (mod 2^63) is x."""
    ginv = pow(G, -1, 1 << M)
    for _ in range(k):
        x = ((x - CC) * ginv) % (1 << M)
    return x


def test_doubled_state_follows_the_recurrence():
    # 2 (g x + c) = g (2x) + 2c mod 2^64, and 2x mod 2^64 keeps the 63 state
    # bits, so z >> 1 is the m-bit state and z >> 11 its top 53 bits
    rng = np.random.default_rng(11)
    for x in rng.integers(0, 2**63, 2000, dtype=np.uint64):
        x = int(x)
        z = (x << 1) & M64
        x1 = (G * x + CC) & M64
        z1 = (G * z + 2 * CC) & M64
        assert z1 >> 1 == x1 & MASK
        assert z1 >> 11 == (x1 & MASK) >> (M - 53)


@pytest.mark.parametrize("draws", [1, 2, 7, 64, 65])
def test_summed_form_equals_per_draw_digest(oracle, draws):
    seeds = oracle.seed_hash(M, 42, 0, 300)
    st, _, dg = oracle.lcg_draw(M, G, CC, seeds, draws, want_u=False)
    for k, x0 in enumerate(seeds):
        x, d, marked = summed_digest(int(x0), draws)
        assert not marked
        assert x == int(st[k]) and d == int(dg[k])


def test_summed_form_at_every_shift(oracle):
    # first draws with every normalising shift 0..31, and the boundary of
    # the zero high word (states 2^31 - 1 and 2^31 of the m-bit recurrence)
    firsts = [(1 << (62 - s)) + 12345 for s in range(32)] + [2**31, 2**31 + 1, 2**32 - 1, 2**62 - 1]
    pre = np.array([start_before(x) for x in firsts], dtype=np.uint64)
    st, _, dg = oracle.lcg_draw(M, G, CC, pre, 3, want_u=False)
    seen = set()
    for k, x0 in enumerate(pre):
        z1 = ((G * ((int(x0) << 1) & M64)) + 2 * CC) & M64
        seen.add(clz32(z1 >> 32))
        x, d, marked = summed_digest(int(x0), 3)
        assert not marked
        assert x == int(st[k]) and d == int(dg[k])
    assert seen >= set(range(32))


def test_zero_high_word_is_marked(oracle):
    # first states below 2^31 have a zero high word in the doubled state;
    # the kernel redoes those streams per draw, so the summed form needs only
    # to mark them
    pre = np.array([start_before(x) for x in (0, 1, 2**20, 2**31 - 1)], dtype=np.uint64)
    for x0 in pre:
        assert summed_digest(int(x0), 4)[2]


def _count_add(acc, s):
    """fp32 add of the subnormal with bit pattern s (round to nearest)."""
    return np.float32(acc + np.array([s], dtype=np.uint32).view(np.float32)[0])


def test_fp32_count_is_exact_and_marks_all_ones():
    # sums of subnormal patterns are exact while below 2^24 units: the
    # kernel's 64-draw sum is at most 64 * 31, and the run-time form folds
    # every 16 draws
    rng = np.random.default_rng(5)
    with np.errstate(all="ignore"):
        for _ in range(200):
            ss = rng.integers(0, 32, 64)
            acc = np.float32(0.0)
            for s in ss:
                acc = _count_add(acc, int(s))
            assert int(np.array([acc], dtype=np.float32).view(np.uint32)[0]) == int(ss.sum())
        worst = np.float32(0.0)
        for _ in range(64):
            worst = _count_add(worst, 31)
        assert int(np.array([worst], dtype=np.float32).view(np.uint32)[0]) == 64 * 31
        marked = _count_add(np.float32(0.0), 5)
        marked = _count_add(marked, 0xFFFFFFFF)
        marked = _count_add(marked, 7)
        bits = int(np.array([marked], dtype=np.float32).view(np.uint32)[0])
        assert np.isnan(marked) and (bits & 0x7FFFFFFF) > 0x7F800000

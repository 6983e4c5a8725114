"""Pins of the oracle's hash (Section 4, Listing 1) and the seeds built on it
(Eqs. 3-5), by inverting the hash with the constants the listing prints:
subhash is a bijection of 64-bit words (odd multiplier; an xor-shift by 47
undoes itself because 2*47 >= 64), so hash(., s) must invert to the key.
A wrong constant, shift or composition order breaks the inversion."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
MASK64 = 2**64 - 1


def _consts():
    d = {}
    with open(os.path.join(HERE, "golden", "listing1_constants.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                d[k] = int(v, 0)
    return d


C = _consts()
MUL, SHIFT, XORMUL = C["M"], C["SHIFT"], C["SEED_XOR_MULTIPLIER"]
MUL_INV = pow(MUL, -1, 2**64)


def unsubhash(y):
    t = y ^ (y >> SHIFT)          # undoes t ^ (t >> 47)
    return (t * MUL_INV) & MASK64  # undoes the multiplication by M


def unhash(h, s, oracle):
    seed_hash = oracle.subhash(s ^ ((XORMUL * MUL) & MASK64))
    sk = ((unsubhash(h) ^ seed_hash) * MUL_INV) & MASK64  # = subhash(k)
    return unsubhash(sk)


def test_subhash_inverts(oracle):
    rng = np.random.default_rng(10)
    for x in [0, 1, MASK64] + [int(v) for v in rng.integers(0, 2**63, size=2000, dtype=np.int64)]:
        assert unsubhash(oracle.subhash(x)) == x


def test_hash_inverts_to_key(oracle):
    rng = np.random.default_rng(11)
    keys = [0, 1, 2, 2**26 - 1, MASK64] + [int(v) for v in rng.integers(0, 2**62, size=500)]
    for s in (0, 42, 7, MASK64):
        for k in keys:
            assert unhash(oracle.hash64(k, s), s, oracle) == k


def test_hash_seed_masks_to_m_bits(oracle):
    for k in range(20):
        h = oracle.hash64(k, 42)
        assert oracle.hash_seed(k, 42, 63) == h & (2**63 - 1)
        assert oracle.hash_seed(k, 42, 64) == h


def test_hash_seeds_unique_over_2_24_ids(oracle):
    # A bijection in k: no two of the 2^24 history ids share a 64-bit seed.
    s = np.sort(oracle.seed_hash(64, 42, 0, 2**24))
    assert not np.any(s[1:] == s[:-1])
    # 63-bit masking: expected colliding pairs ~ n^2 / 2^64 = 2^-16.
    s63 = np.sort(oracle.seed_hash(63, 42, 0, 2**24))
    assert np.count_nonzero(s63[1:] == s63[:-1]) <= 1


def test_hash_avalanche(oracle):
    # Flipping one key bit flips about half of the 64 output bits.
    rng = np.random.default_rng(12)
    flips = []
    for k in (int(v) for v in rng.integers(0, 2**62, size=64)):
        h = oracle.hash64(k, 42)
        for b in range(64):
            flips.append(bin(h ^ oracle.hash64(k ^ (1 << b), 42)).count("1"))
    mean = np.mean(flips)
    assert 30.0 < mean < 34.0


def test_hierarchical_seed_is_two_hashes(oracle):
    # Eq. (4): S_{i,j} = hash(j, hash(i, s)); different batches i give
    # unrelated seeds for the same particle index j.
    s = 42
    for i in range(4):
        parent = oracle.hash64(i, s)
        for j in range(4):
            h = oracle.hash64(j, parent)
            assert unhash(h, parent, oracle) == j
    row0 = set(int(v) for v in oracle.seed_hash(64, oracle.hash64(0, s), 0, 4096))
    row1 = set(int(v) for v in oracle.seed_hash(64, oracle.hash64(1, s), 0, 4096))
    assert not (row0 & row1)


@pytest.mark.parametrize("s", [42, 7])
def test_hash_key_order_fixed(oracle, s):
    # hash(k, s) != hash(s, k) in general: key and seed play different roles.
    assert oracle.hash64(3, s) != oracle.hash64(s, 3)

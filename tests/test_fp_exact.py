"""The fp64 steps the transport computes on the integer pipes, evaluated on
the host through the C ABI, against the host's IEEE arithmetic: the
reciprocal must equal 1/y (division rounded to nearest even) bit for bit,
and 2u - 1 must equal the fp64 expression 2.0 * u - 1.0 for u = n 2^-53."""
import math
import random
import struct

import numpy as np
import pytest


@pytest.fixture(scope="module")
def mc():
    from paper_2403_06362_gb300 import _build
    _build.build()
    import paper_2403_06362_gb300 as mc
    mc.lib()
    return mc


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def from_bits(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def recip_inputs():
    rng = random.Random(105)
    ys = []
    for _ in range(200000):  # random mantissas over a wide exponent range
        ys.append(from_bits((rng.randrange(1, 2047 - 4) << 52) | rng.getrandbits(52)))
    for m in [1, 2, 3, (1 << 52) - 1, (1 << 52) - 2, (1 << 51), (1 << 51) + 1, 0x5555555555555, 0xAAAAAAAAAAAAA]:
        for e in (1, 2, 500, 1023, 1500, 2043, 2044):
            ys.append(from_bits((e << 52) | m))
    for n in range(1, 3000):  # mantissas near 1 and near 2
        ys.append(from_bits((1023 << 52) | n))
        ys.append(from_bits((1023 << 52) | ((1 << 52) - n)))
    for j in range(1024):  # mantissas on and next to the edges of the 1024 cells of [1, 2)
        for d in (0, 1, 2, (1 << 42) - 1, (1 << 42) - 2):
            m = (j << 42) + d
            if 0 < m < (1 << 52):
                ys.append(from_bits((1022 << 52) | m))
    ys += [2.0**k for k in range(-1020, 1021, 7)]
    ys += [(2 * n - 2**53) * 2.0**-53 for n in range(1, 4000) if n != 2**52]  # slab directions
    ys += [-y for y in ys[:50000]]
    return ys


def test_reciprocal_equals_ieee_division(mc):
    bad = [(y.hex(), mc.mc_recip_rn(y).hex(), (1.0 / y).hex()) for y in recip_inputs()
           if bits(mc.mc_recip_rn(y)) != bits(1.0 / y)]
    assert not bad, bad[:5]


def test_reciprocal_edge_cases_fall_back(mc):
    for y in (5e-324, 2.0**-1030, 1.7e308, -2.0**1023, float("inf")):
        assert bits(mc.mc_recip_rn(y)) == bits(1.0 / y)


def test_two_u_minus_1_equals_the_fp64_expression(mc):
    rng = random.Random(53)
    ns = [rng.getrandbits(53) for _ in range(100000)]
    ns += [0, 1, 2, 3, 2**52 - 1, 2**52, 2**52 + 1, 2**53 - 1, 2**53 - 2, 2**51, 3 * 2**51]
    ns += [rng.getrandbits(k) for k in range(1, 53) for _ in range(50)]
    for n in ns:
        u = n * 2.0**-53
        assert bits(mc.mc_two_u_minus_1(n)) == bits(2.0 * u - 1.0), n


def test_llrint_nonneg_rounds_half_to_even(mc):
    rng = random.Random(62)
    vs = [rng.random() * 2.0 ** rng.randrange(-3, 62) for _ in range(100000)]
    vs += [k + 0.5 for k in range(0, 50)] + [0.0, 0.49999999999999994, 0.5, 1.5, 2.5, 2.0**52 + 1, 2.0**61]
    vs += [(2 * k + 1) * 2.0**-e for e in range(1, 40) for k in range(5)]
    for v in vs:
        assert mc.lib().mc_llrint_nonneg(v) == round(v), v  # Python's round: half to even


def test_order_keys_compare_like_doubles(mc):
    rng = random.Random(64)
    special = [0.0, -0.0, 5e-324, -5e-324, 1.0, -1.0, 2.0**-1022, -(2.0**-1022), 1.7e308, -1.7e308]
    xs = special + [rng.uniform(-1, 1) * 2.0 ** rng.randrange(-60, 60) for _ in range(3000)]
    for i in range(0, len(xs) - 1):
        for a, b in ((xs[i], xs[i + 1]), (xs[i + 1], xs[i]), (xs[i], xs[i])):
            assert mc.lib().mc_d_lt(a, b) == int(a < b), (a, b)
    for a in special:
        for b in special:
            assert mc.lib().mc_d_lt(a, b) == int(a < b), (a, b)


def test_small_integer_products_round_once(mc):
    rng = random.Random(11)
    hs = [rng.uniform(0.001, 1000.0) for _ in range(3000)] + [100.0 / 64, 0.1, 1.0 / 3, 2.0**-20, 1.5625]
    for h in hs:
        for j in [0, 1, 2, 3, 7, 63, 64, 65, 1023, 2047] + [rng.randrange(2048) for _ in range(10)]:
            assert bits(mc.mc_mul_small(j, h)) == bits(float(j) * h), (j, h)


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

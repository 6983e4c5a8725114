"""The fp64 flight logarithm ln(1 - u) (table-driven, Tang 1990) evaluated on
the host through the C ABI, against ln(1 - u) computed to 40 significant
digits with Python's decimal module and rounded once.  Every uniform of the
library is a multiple of 2^-53 in [0, 1), so those are the inputs: uniform,
log-uniform over every binade down to 2^-53, and the edges of the two
branches and of the 1024 table cells."""
import math
import random
from decimal import Decimal, getcontext

import pytest


@pytest.fixture(scope="module")
def mc():
    from paper_2403_06362_gb300 import _build
    _build.build()
    import paper_2403_06362_gb300 as mc
    mc.lib()
    return mc


def exact(u: float) -> Decimal:
    getcontext().prec = 40
    return (Decimal(1) - Decimal(u)).ln()


def ulp_error(y: float, u: float) -> float:
    ref = exact(u)
    r = float(ref)
    return float(abs(Decimal(y) - ref) / Decimal(math.ulp(r))) if r != 0.0 else abs(y) / 5e-324


def inputs():
    rng = random.Random(2403)
    us = [rng.getrandbits(53) * 2.0**-53 for _ in range(6000)]
    for e in range(1, 54):  # every binade [2^-e, 2^-e+1)
        us += [(2**(53 - e) + rng.getrandbits(53 - e)) * 2.0**-53 for _ in range(40)]
    us += [2.0**-53, 2.0**-8 - 2.0**-53, 2.0**-8, 2.0**-8 + 2.0**-53, 0.5, 1.0 - 2.0**-53, 1.0 - 2.0**-52]
    for j in range(1025):  # x = 1 - u on the edges of the 1024 table cells, in a few binades
        for k in (1, 4, 30):
            x = (1.0 + j / 1024.0) * 2.0**-k
            if 0.0 < x < 1.0:
                us += [1.0 - x, 1.0 - x - 2.0**-53, 1.0 - x + 2.0**-53]
    return [u for u in us if 0.0 < u < 1.0]


def test_zero_gives_zero(mc):
    assert math.copysign(1.0, mc.mc_log1m(0.0)) == 1.0 and mc.mc_log1m(0.0) == 0.0


def test_within_one_ulp_of_correctly_rounded(mc):
    worst = 0.0
    for u in inputs():
        err = ulp_error(mc.mc_log1m(u), u)
        worst = max(worst, err)
        assert err < 1.0, (u.hex(), err)
    assert worst > 0.5  # the test does measure something


def test_table_branch_within_a_hair_of_correct_rounding(mc):
    # u >= 2^-8: the fixed-point sum is accurate to about 2^-68 against a
    # result of at least 2^-8 (an ulp of at least 2^-60), so the rounding can
    # miss only by a small fraction of an ulp past the halfway point
    worst = max(ulp_error(mc.mc_log1m(u), u) for u in inputs() if u >= 2.0**-8)
    assert worst < 0.5005, worst


def test_mostly_correctly_rounded(mc):
    # glibc's log is correctly rounded in all but rare cases; the table log
    # agrees with it on the large majority of inputs
    us = inputs()
    same = sum(mc.mc_log1m(u) == math.log(1.0 - u) for u in us)
    assert same >= 0.95 * len(us)


def test_monotone_on_a_dense_run(mc):
    # ln(1 - u) must not increase along consecutive multiples of 2^-53,
    # across the branch switch at 2^-8 and across a table cell edge
    for start in (2.0**-8 - 300 * 2.0**-53, 1.0 - (1.0 + 64 / 128.0) * 0.5 - 300 * 2.0**-53):
        prev = mc.mc_log1m(start)
        for i in range(1, 600):
            y = mc.mc_log1m(start + i * 2.0**-53)
            assert y <= prev
            prev = y


def test_committed_tables_are_the_generated_ones():
    import importlib.util
    import os
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2403_06362_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("gen_log_table", os.path.join(csrc, "gen_log_table.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    with open(os.path.join(csrc, "log_table.inc")) as f:
        assert f.read() == gen.render()

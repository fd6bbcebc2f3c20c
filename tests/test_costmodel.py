"""The cost-model components against closed forms and brute-force expectations."""
import itertools
import math
from fractions import Fraction

import pytest

from paper_1311_0059_gb300 import costmodel as cm


def test_yao_boundaries():
    assert cm.i_key(0, 1000, 10) == 0
    assert cm.i_key(1000, 1000, 10) == pytest.approx(10)
    assert cm.i_raw(0, 1000, 10) == 0
    assert cm.i_raw(10, 1000, 10) == pytest.approx(1000)


@pytest.mark.parametrize("r", [1, 17, 250, 600])
def test_i_raw_inverts_i_key(r):
    n, m = 1000, 370
    assert cm.i_raw(cm.i_key(r, n, m), n, m) == pytest.approx(r, rel=1e-9)


def test_expected_distinct_by_enumeration():
    # exact mean of the number of distinct values over all U**n sequences
    for u, n in [(3, 4), (4, 3), (5, 5), (2, 6)]:
        tot = sum(len(set(seq)) for seq in itertools.product(range(u), repeat=n))
        exact = Fraction(tot, u ** n)
        assert cm.expected_distinct(u, n) == pytest.approx(float(exact), rel=1e-12)


def test_generator_size_inverts():
    for m, n in [(500, 2000), (49_000_000, 200_000_000)]:
        u = cm.generator_size(m, n)
        assert cm.expected_distinct(u, n) == pytest.approx(m, rel=1e-9)


def test_eq1_satisfies_its_definition():
    # M - P = G*F - (M - 1) * P
    for g, m, f in [(1000, 64, 1.2), (5e6, 4096, 1.0), (3e4, 100, 1.6)]:
        p = cm.eq1_partitions(g, m, f)
        assert m - p == pytest.approx(g * f - (m - 1) * p)


def test_prepartition_io():
    assert cm.prepartition_io(100, 50, 50) == 100         # all groups resident: no spill
    assert cm.prepartition_io(100, 0, 50) == 200          # nothing resident: everything spills
    assert cm.predicted_spill_records(200e6, 2e6, 49e6) == pytest.approx(200e6 * (1 - 2 / 49))
    assert cm.grace_io(2, 10) == 40


def test_estimate_groups_recovers_g():
    n, g, k = 200e6, 49e6, 2e6
    r_h = cm.i_raw(k, n, g)
    assert cm.estimate_groups(r_h, k, n) == pytest.approx(g, rel=1e-6)

"""The paper's cost-model components used for planning and reporting.

* Input component (Appendix A.1, Yao's formula):
  I_key(r, n, m) = m * (1 - (1 - r/n)**(n/m))  - distinct keys in r of n records
  I_raw(k, n, m) = n * (1 - (1 - k/m)**(m/n))  - records drawn to see k keys
* Generator-set size (Appendix A.4): the expected number of distinct keys in n
  draws with replacement from U keys is U * (1 - (1 - 1/U)**n).
* Eq. 1 (Section 4.3): spilled partitions P = (G*F - M) / (M - 2).
* Pre-Partitioning I/O (Section 5.3.4): C_IO = R + (R - K/G_t * R); the second
  term is the spilled share of the input, so the predicted spill of raw records
  is R_t * (1 - K/G_t) records when K < G_t (else 0).
* Grace partitioning (Section 5.3): L levels cost 2*L*R I/O.

Every function is plain float arithmetic on the formulas as printed.
"""
from __future__ import annotations

import math


def i_key(r: float, n: float, m: float) -> float:
    if n <= 0 or m <= 0:
        return 0.0
    r = min(max(r, 0.0), n)
    return m * (1.0 - (1.0 - r / n) ** (n / m))


def i_raw(k: float, n: float, m: float) -> float:
    if n <= 0 or m <= 0:
        return 0.0
    k = min(max(k, 0.0), m)
    return n * (1.0 - (1.0 - k / m) ** (m / n))


def expected_distinct(u: float, n: float) -> float:
    """U * (1 - (1 - 1/U)**n): mean distinct keys in n draws from U keys."""
    if u <= 0:
        return 0.0
    return u * (1.0 - math.exp(n * math.log1p(-1.0 / u))) if u > 1 else (1.0 if n > 0 else 0.0)


def generator_size(m: float, n: float) -> float:
    """Solves expected_distinct(U, n) = m for U (bisection)."""
    if m <= 0 or n <= 0:
        return 0.0
    if m >= n:
        return math.inf
    lo, hi = m, m
    while expected_distinct(hi, n) < m:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if expected_distinct(mid, n) < m:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def eq1_partitions(g: float, m: float, fudge: float = 1.2) -> float:
    """Eq. 1: P = (G*F - M) / (M - 2), G and M in frames."""
    return (g * fudge - m) / (m - 2.0)


def prepartition_io(r: float, k: float, g_t: float) -> float:
    """C_IO of Pre-Partitioning (Section 5.3.4) in the unit of r."""
    frac = min(k / g_t, 1.0) if g_t > 0 else 1.0
    return r + (r - frac * r)


def predicted_spill_records(r_t: float, k: float, g_t: float) -> float:
    """Raw records the Pre-Partitioning model spills at level 0: R_t(1 - K/G_t)."""
    return prepartition_io(r_t, k, g_t) - r_t


def grace_io(levels: int, r: float) -> float:
    return 2.0 * levels * r


def estimate_groups(rows_at_full: float, k: float, n: float) -> float:
    """Estimate of G_t from the fill point of the table: the table held K groups
    after R_H rows, and R_H = I_raw(K, n, G) (Appendix A.1); solved for G."""
    if rows_at_full <= 0 or rows_at_full >= n or k <= 0:
        return k
    lo, hi = k, max(k * 2.0, 2.0)
    while i_raw(k, n, hi) > rows_at_full and hi < 1e18:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if i_raw(k, n, mid) > rows_at_full:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)

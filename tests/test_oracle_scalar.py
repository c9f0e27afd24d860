"""Pins of the oracle's scalar update forms to the paper and to exact arithmetic.

* Tables 1 and 2 (printed FP64 values of d-tilde and d-hat) reproduce bit for bit.
* d-bar lies within a few ulps of the exact real root (80-digit decimal).
* The two independent d-bar searches (ulp walk, bit-pattern bisection) agree.
* d-bar is monotone where d-tilde and d-hat are not (section "Achieving Exact
  Monotonicity"), and causal in the sense of the paper's definition.
"""
import math

import numpy as np
import pytest

import oracle
from tests.oracle_pins import (INF, check_dbar_against_exact_root, exact_root, read_table,
                               ulps_from)


def test_table1_dtilde_reproduces_bit_exactly():
    rows = read_table("table1_dtilde.txt")
    for case, v, h, tH, tV, expect in rows:
        got = oracle.dtilde(v, h, tH, tV)
        assert got == expect, (case, got, expect)
    (_, _, _, _, tVA, dA), (_, _, _, _, tVB, dB) = rows
    assert tVB < tVA and dB > dA      # the non-monotonicity the table shows


def test_table2_dhat_reproduces_bit_exactly():
    rows = read_table("table2_dhat.txt")
    for case, v, h, tH, tV, expect in rows:
        got = oracle.dhat(v, h, tH, tV)
        assert got == expect, (case, got, expect)
    (_, _, _, _, tVA, dA), (_, _, _, _, tVB, dB) = rows
    assert tVB < tVA and dB > dA


def test_cell_constant_rounding():
    # c = fl(fl(h/v)^2): on the Table 2 cell this differs from fl(h*h)/fl(v*v).
    v, h = 1500.0, 1.25
    assert oracle.cell_c(v, h) == (h / v) * (h / v)
    assert oracle.cell_c(v, h) != (h * h) / (v * v)


@pytest.mark.parametrize("table", ["table1_dtilde.txt", "table2_dhat.txt"])
def test_dbar_monotone_on_the_tables(table):
    rows = read_table(table)
    (_, v, h, tH, tVA, _), (_, _, _, _, tVB, _) = rows
    r = h / v
    c = oracle.cell_c(v, h)
    dA = oracle.dbar([tH, tVA], r, c)
    dB = oracle.dbar([tH, tVB], r, c)
    assert tVB < tVA and dB <= dA
    # and it is the correctly placed root of the same equation
    for tV, d in ((tVA, dA), (tVB, dB)):
        assert ulps_from(d, exact_root([tH, tV], c)) <= 2.0


def test_dbar_within_ulps_of_exact_root():
    worst = check_dbar_against_exact_root(lambda a, r, c: oracle.dbar(a, r, c))
    assert worst <= 2.0


def test_dbar_two_searches_agree():
    rng = np.random.Generator(np.random.PCG64(7))
    from tests.oracle_pins import random_minima
    for i in range(3000):
        D = 2 + (i % 2)
        a, r = random_minima(rng, D)
        c = r * r
        assert oracle.dbar(a, r, c) == oracle.dbar_bisect(a, c), (a, r)


def _neighbourhood(x, k):
    out = [x]
    up = dn = x
    for _ in range(k):
        up = math.nextafter(up, INF)
        dn = math.nextafter(dn, -INF)
        out += [up, dn]
    return sorted(out)


@pytest.mark.parametrize("table", ["table1_dtilde.txt", "table2_dhat.txt"])
def test_dbar_monotone_exhaustive_near_tables(table):
    rows = read_table(table)
    _, v, h, tH, tV, _ = rows[0]
    r = h / v
    c = oracle.cell_c(v, h)
    tHs = _neighbourhood(tH, 64)      # every pair within +-64 ulps of the table's inputs
    tVs = _neighbourhood(tV, 64)
    grid = np.array([[oracle.dbar([x, y], r, c) for y in tVs] for x in tHs])
    assert np.all(np.diff(grid, axis=0) >= 0.0)
    assert np.all(np.diff(grid, axis=1) >= 0.0)
    # d-hat on the same neighbourhood is not monotone (the paper's point)
    hat = np.array([[oracle.dhat(v, h, x, y) for y in tVs] for x in tHs])
    if table == "table2_dhat.txt":
        assert np.any(np.diff(hat, axis=1) < 0.0)


def test_dbar_monotone_random():
    rng = np.random.Generator(np.random.PCG64(3))
    from tests.oracle_pins import random_minima
    for i in range(2000):
        D = 2 + (i % 2)
        a, r = random_minima(rng, D)
        c = r * r
        d0 = oracle.dbar(a, r, c)
        k = int(rng.integers(D))
        if a[k] == INF:
            continue
        lowered = list(a)
        lowered[k] = max(0.0, a[k] - float(rng.choice([0.0, 1e-15, 1e-9, 1e-3])) * max(a[k], 1e-300)
                         - math.ulp(a[k]) * int(rng.integers(0, 4)))
        assert oracle.dbar(lowered, r, c) <= d0


def test_dbar_special_cases():
    r = 2.0 ** -7
    c = r * r
    assert oracle.dbar([INF, INF], r, c) == INF
    assert oracle.dbar([INF, INF, INF], r, c) == INF
    # one finite neighbour, dyadic numbers: one-sided update is exact
    for k in range(0, 300, 7):
        a = k * r
        assert oracle.dbar([a, INF], r, c) == (k + 1) * r
        assert oracle.dbar([INF, a, INF], r, c) == (k + 1) * r
    # the result is strictly above the smallest neighbour (causality needs it)
    rng = np.random.Generator(np.random.PCG64(5))
    from tests.oracle_pins import random_minima
    for i in range(500):
        a, rr = random_minima(rng, 2 + i % 2)
        assert oracle.dbar(a, rr, rr * rr) > min(a)


def test_dbar_causal():
    """Changing a neighbour whose value is at or above the result leaves the
    result unchanged (the causality definition: only the upwind set counts)."""
    rng = np.random.Generator(np.random.PCG64(9))
    from tests.oracle_pins import random_minima
    for i in range(1000):
        D = 2 + i % 2
        a, r = random_minima(rng, D)
        c = r * r
        d = oracle.dbar(a, r, c)
        for k in range(D):
            if a[k] >= d:
                for nv in (d, d * 1.5 + 1.0, INF):
                    b = list(a)
                    b[k] = nv
                    assert oracle.dbar(b, r, c) == d


def test_dbar_symmetric_in_2d():
    rng = np.random.Generator(np.random.PCG64(13))
    from tests.oracle_pins import random_minima
    for _ in range(1000):
        a, r = random_minima(rng, 2)
        c = r * r
        assert oracle.dbar(a, r, c) == oracle.dbar(a[::-1], r, c)

"""Pins of the explicit update forms of the Mitigation Strategies section
(Algorithm 1 with the classical root d-tilde or the rearranged root d-hat) and
of the form-aware Table 3 residual, against what the paper prints and what the
mathematics fixes: Tables 1 and 2, exact real roots, the one-sided closed form,
the case boundary and hand-built residual cases."""
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
import synth
from tests.oracle_pins import INF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out.append((f[0], *map(float, f[1:])))
    return out


@pytest.mark.parametrize("form,table", [(1, "table1_dtilde.txt"), (2, "table2_dhat.txt")])
def test_tables_through_the_update(form, table):
    for case, v, h, tH, tV, want in _rows(table):
        got = oracle.update_form(form, v, h, tH, tV)
        assert got == want, (case, got, want)
        assert oracle.update_form(form, v, h, tV, tH) == want      # symmetric in tH, tV


def test_tables_show_the_loss_of_monotonicity():
    (_, v, h, tH, tVa, da), (_, _, _, _, tVb, db) = _rows("table1_dtilde.txt")
    assert tVb < tVa and oracle.update_form(1, v, h, tH, tVb) > oracle.update_form(1, v, h, tH, tVa)
    # d-bar keeps order on the same inputs
    assert oracle.update_form(0, v, h, tH, tVb) <= oracle.update_form(0, v, h, tH, tVa)


def _exact_2d(tH, tV, r) -> Decimal:
    getcontext().prec = 80
    a, b, R = Decimal(tH), Decimal(tV), Decimal(r)
    c = R * R
    return (a + b + (2 * c - (a - b) ** 2).sqrt()) / 2


def test_quadratic_roots_are_close_to_the_exact_root():
    rng = np.random.Generator(np.random.PCG64(3))
    worst = {1: 0.0, 2: 0.0}
    for _ in range(2000):
        v = float(rng.uniform(0.5, 4.0))
        h = float(rng.choice([1.0, 0.25, 4.0]))
        r = h / v
        tH = float(rng.uniform(0.0, 50.0))
        tV = tH + float(rng.uniform(-0.95, 0.95)) * r
        if abs(tH - tV) >= r:
            continue
        # the rounding of r and c only perturbs the root within a few ulps
        ex = _exact_2d(tH, tV, r * 1.0)
        for form in (1, 2):
            got = oracle.update_form(form, v, h, tH, tV)
            err = float(abs(Decimal(got) - ex) / ex)
            worst[form] = max(worst[form], err)
    assert worst[2] < 1e-14          # d-hat: a few ulps
    assert worst[1] < 1e-9           # d-tilde: cancellation, still far below the step


def test_one_sided_case_and_boundary():
    v, h = 2.0, 1.0
    r = h / v
    for form in (1, 2):
        assert oracle.update_form(form, v, h, 3.0, 3.0 + r) == 3.0 + r          # |d| == r: one-sided
        assert oracle.update_form(form, v, h, 3.0 + 2 * r, 3.0) == 3.0 + r      # |d| > r
        assert oracle.update_form(form, v, h, 3.0, INF) == 3.0 + r
        assert oracle.update_form(form, v, h, INF, 7.0) == 7.0 + r
        assert oracle.update_form(form, v, h, INF, INF) == INF
        assert 3.0 + r / 2 < oracle.update_form(form, v, h, 3.0, 3.0 + r / 2) < 3.0 + r


def test_residual_form_on_a_line():
    # 1 x 4 line, source at 0, v = 1, h = 1/8: one-sided updates only, exact
    speed = np.ones((1, 4))
    h = 0.125
    t = np.array([[0.0, 0.125, 0.25, 0.375]])
    for form in (0, 1, 2):
        assert oracle.residual(speed, h, [0], t, form=form) == (0, 0.0)
    bad = t.copy()
    bad[0, 3] = math.nextafter(0.375, 1.0)
    for form in (0, 1, 2):
        n, rel = oracle.residual(speed, h, [0], bad, form=form)
        assert n == 1 and rel == (bad[0, 3] - 0.375) / bad[0, 3]


def test_residual_form_counts_a_quadratic_cell():
    # 2 x 2, source at (0,0): cells (0,1), (1,0) one-sided; (1,1) quadratic
    speed = np.ones((2, 2))
    h = 1.0
    t = np.array([[0.0, 1.0], [1.0, 0.0]])
    for form in (1, 2):
        t[1, 1] = oracle.update_form(form, 1.0, h, 1.0, 1.0)
        assert oracle.residual(speed, h, [0], t, form=form) == (0, 0.0)
        # (1 + 1 + sqrt(2)) / 2 within rounding
        assert abs(t[1, 1] - (1.0 + math.sqrt(0.5))) < 1e-15
        t2 = t.copy()
        t2[1, 1] = math.nextafter(t[1, 1], 0.0)
        assert oracle.residual(speed, h, [0], t2, form=form)[0] == 1


def test_residual_of_the_exact_fixed_point_under_the_explicit_forms_is_small():
    p = synth.random_problem(9, (40, 50), n_src=2, contrast=4.0, smooth_sigma=2.0, h=1.0)
    t = oracle.fmm(p.speed, p.h, p.sources).t
    assert oracle.residual(p.speed, p.h, p.sources, t) == (0, 0.0)
    for form in (1, 2):
        n, rel = oracle.residual(p.speed, p.h, p.sources, t, form=form)
        assert rel < 1e-12            # d-bar and the explicit roots agree to rounding


def test_residual_form_rejects_3d():
    speed = np.ones((3, 3, 3))
    t = np.zeros((3, 3, 3))
    with pytest.raises(RuntimeError):
        oracle.residual(speed, 1.0, [0], t, form=1)


def _ulp_scale(tau, tH, tV):
    # the update rounds tau - tH and tau - tV: its error is relative to the
    # largest magnitude among tau, the minima and those differences
    return math.ulp(max(abs(tau), abs(tH), abs(tV), abs(tau - tH), abs(tau - tV)))


def test_newton_variant_close_to_the_exact_root():
    """Form 3 (d-hat, then Newton's method on alpha = 0) lands within 2 ulps (of
    the largest magnitude in the update) of the exact root of the quadratic with
    the same c, over scales from 1e-3 to 1e3 and minima of either sign."""
    getcontext().prec = 80
    rng = np.random.Generator(np.random.PCG64(7))
    n = 0
    for _ in range(4000):
        v = float(rng.uniform(0.5, 4.0))
        h = float(rng.choice([1.0, 0.25, 4.0]))
        r = h / v
        tH = float(rng.uniform(0.0, 50.0)) * float(rng.choice([1e-3, 1.0, 1e3]))
        tV = tH + float(rng.uniform(-0.95, 0.95)) * r
        if abs(tH - tV) >= r:
            continue
        c = Decimal(r * r)
        a, b = Decimal(tH), Decimal(tV)
        root = (a + b + (2 * c - (a - b) ** 2).sqrt()) / 2
        got = oracle.update_form(3, v, h, tH, tV)
        assert abs(Decimal(got) - root) <= 2 * Decimal(_ulp_scale(got, tH, tV)), (v, h, tH, tV, got)
        n += 1
    assert n > 3000


@pytest.mark.parametrize("table,broken", [("table1_dtilde.txt", 1), ("table2_dhat.txt", 2)])
def test_newton_variant_orders_the_table_pairs(table, broken):
    """The paper reports the Newton variant deterministic in its tests: on the two
    input pairs of Tables 1 and 2, where d-tilde and d-hat respectively lose
    monotonicity, form 3 keeps the order of its inputs."""
    (_, v, h, tH, tVa, _), (_, _, _, _, tVb, _) = _rows(table)
    assert tVb < tVa
    assert oracle.update_form(broken, v, h, tH, tVb) > oracle.update_form(broken, v, h, tH, tVa)
    assert oracle.update_form(3, v, h, tH, tVb) <= oracle.update_form(3, v, h, tH, tVa)


def test_newton_variant_one_sided_and_symmetric():
    rng = np.random.Generator(np.random.PCG64(8))
    for _ in range(500):
        v = float(rng.uniform(0.5, 4.0))
        h = float(rng.choice([1.0, 0.5, 2.0]))
        r = h / v
        tH = float(rng.uniform(0.0, 20.0))
        tV = tH + float(rng.choice([-1.0, 1.0])) * float(rng.uniform(1.0, 3.0)) * r
        assert oracle.update_form(3, v, h, tH, tV) == min(tH, tV) + r      # one-sided
        tV2 = tH + float(rng.uniform(-0.9, 0.9)) * r
        assert oracle.update_form(3, v, h, tH, tV2) == oracle.update_form(3, v, h, tV2, tH)
    assert oracle.update_form(3, 1.0, 1.0, INF, 2.0) == 3.0
    assert oracle.update_form(3, 1.0, 1.0, INF, INF) == INF


def test_upsampled_input_keeps_the_physical_problem():
    """Table 3's x4 input (nearest-neighbour upsampling by 4 per axis, h / 4): on a
    constant-speed grid with one source the upsampled solve's axis values are the
    original ones at the same physical points, k h exactly along the source row."""
    p = synth.Problem("c", np.ones((6, 9)), 1.0, np.array([4], dtype=np.int64), np.zeros(1))
    q = synth.upsampled(p, 4)
    assert q.speed.shape == (24, 36) and q.h == 0.25 and list(q.sources) == [16]
    t = oracle.fmm(q.speed, q.h, q.sources).t
    assert np.array_equal(t[0], np.abs(np.arange(36) - 16) * 0.25)
    assert np.array_equal(synth.upsampled(p, 4).speed[::4, ::4], p.speed)

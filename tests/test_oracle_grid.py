"""Pins of the oracle's grid solvers.

* Closed forms: plane waves and the axes through a point source at constant
  speed and dyadic spacing are exactly k*h; every step of a 1D line with random
  speeds sits within a few ulps of the exact real one-step root.
* Theorem 1: the fast marching method (Algorithm 2), the topology-driven
  solver (Algorithm 4), the fast sweeping method (Algorithm 5) and relaxation
  in random orders reach the identical bit pattern.
* The Table 3 residual of that field is exactly 0 and detects a 1-ulp change.
* Invariants: causality, non-negativity, FMM pops in order, no increasing
  update, exact x<->y symmetry, first-order convergence to the continuum.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.oracle_pins import INF, closed_form_axis, exact_root, ulps_from


def test_point_source_axes_exact():
    speed, h, src, m = closed_form_axis(33)
    t = oracle.fmm(speed, h, src).t
    for k in range(-m, m + 1):
        assert t[m, m + k] == abs(k) * h
        assert t[m + k, m] == abs(k) * h


def test_point_source_axes_exact_3d():
    n = 17
    m = n // 2
    h = 2.0 ** -5
    t = oracle.fmm(np.ones((n, n, n)), h, [(m * n + m) * n + m]).t
    for k in range(-m, m + 1):
        assert t[m, m, m + k] == abs(k) * h
        assert t[m, m + k, m] == abs(k) * h
        assert t[m + k, m, m] == abs(k) * h


@pytest.mark.parametrize("shape,axis", [((9, 21), 0), ((21, 9), 1), ((6, 7, 8), 0),
                                        ((6, 7, 8), 2)])
def test_plane_wave_exact(shape, axis):
    h = 2.0 ** -6
    speed = np.ones(shape)
    idx = np.arange(speed.size).reshape(shape)
    src = np.take(idx, 0, axis=axis).ravel()
    t = oracle.fmm(speed, h, src).t
    k = np.arange(shape[axis]).reshape([-1 if d == axis else 1 for d in range(len(shape))])
    assert np.array_equal(t, np.broadcast_to(k * h, shape))


@pytest.mark.parametrize("shape", [(1, 40), (40, 1)])
def test_line_steps_match_exact_roots(shape):
    rng = np.random.Generator(np.random.PCG64(21))
    speed = rng.uniform(1.0, 10.0, shape)
    h = 0.37
    t = oracle.fmm(speed, h, [0]).t.ravel()
    v = speed.ravel()
    assert t[0] == 0.0
    for k in range(1, t.size):
        r = h / v[k]
        ref = exact_root([t[k - 1]], r * r)
        assert ulps_from(t[k], ref) <= 2.0


def test_diagonal_cell_matches_exact_root():
    n = 9
    h = 0.1
    t = oracle.fmm(np.full((n, n), 2.0), h, [4 * n + 4]).t
    r = h / 2.0
    ref = exact_root([t[4, 5], t[5, 4]], r * r)
    assert t[4, 5] == t[5, 4]
    assert ulps_from(t[5, 5], ref) <= 2.0
    # and the exact continuum value of this first diagonal step: r + r/sqrt(2)
    assert abs(t[5, 5] - (r + r / math.sqrt(2.0))) < 1e-15


SMALL = [(2, 2), (3, 5), (1, 7), (7, 1), (17, 13), (12, 12), (5, 5, 5), (3, 4, 6), (2, 9, 3)]


@pytest.mark.parametrize("shape", SMALL)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_all_schedules_reach_the_same_bits(shape, seed):
    nsrc = 1 + seed
    p = synth.random_problem(100 * seed + len(shape), shape, n_src=nsrc, contrast=10.0,
                             src_t_max=0.5 if seed == 2 else 0.0, h=0.25)
    f = oracle.fmm(p.speed, p.h, p.sources, p.src_t)
    g = oracle.sweep(p.speed, p.h, p.sources, p.src_t, mode=0)
    s = oracle.sweep(p.speed, p.h, p.sources, p.src_t, mode=1)
    perm = synth.shuffled_order(seed + 77, p.speed.size)
    r = oracle.relax_order(p.speed, p.h, p.sources, perm, p.src_t)
    for other in (g, s, r):
        assert np.array_equal(f.t.view(np.uint64), other.t.view(np.uint64))
    for st in (f.stats, g.stats, s.stats, r.stats):
        assert st["increases"] == 0
    assert f.stats["order_breaks"] == 0
    bad, mr = oracle.residual(p.speed, p.h, p.sources, f.t, p.src_t)
    assert bad == 0 and mr == 0.0


def _axis_min(t):
    """Smallest neighbour value of every cell (off-grid = +inf)."""
    pad = np.pad(t, 1, constant_values=INF)
    out = np.full(t.shape, INF)
    for ax in range(t.ndim):
        for sh in (-1, 1):
            sl = [slice(1, -1)] * t.ndim
            sl[ax] = slice(1 + sh, pad.shape[ax] - 1 + sh)
            out = np.minimum(out, pad[tuple(sl)])
    return out


@pytest.mark.parametrize("shape", [(31, 29), (11, 12, 13)])
def test_causality_and_sign(shape):
    p = synth.random_problem(5, shape, n_src=3, contrast=10.0, h=1.0)
    t = oracle.fmm(p.speed, p.h, p.sources).t
    src = np.zeros(t.size, bool)
    src[p.sources] = True
    src = src.reshape(shape)
    assert np.all(t >= 0.0) and np.all(np.isfinite(t))
    assert not np.any(np.signbit(t))
    nb = _axis_min(t)
    assert np.all(t[~src] > nb[~src])


def test_xy_symmetry_exact():
    p = synth.random_problem(8, (23, 37), n_src=2, contrast=10.0)
    t = oracle.fmm(p.speed, p.h, p.sources).t
    ny, nx = p.speed.shape
    ys, xs = np.unravel_index(p.sources, (ny, nx))
    srcT = np.ravel_multi_index((xs, ys), (nx, ny))
    tT = oracle.fmm(p.speed.T.copy(), p.h, srcT).t
    assert np.array_equal(t.T, tT)


def test_residual_detects_one_ulp():
    p = synth.random_problem(4, (15, 16), n_src=1, contrast=4.0)
    t = oracle.fmm(p.speed, p.h, p.sources).t
    assert oracle.residual(p.speed, p.h, p.sources, t) == (0, 0.0)
    t2 = t.copy()
    i = np.unravel_index(np.argmax(t), t.shape)
    t2[i] = math.nextafter(t2[i], INF)
    bad, mr = oracle.residual(p.speed, p.h, p.sources, t2)
    assert bad >= 1 and 0.0 < mr < 1e-15


def test_first_order_convergence():
    errs = []
    for n in (33, 65, 129):
        h = 1.0 / (n - 1)
        m = n // 2
        t = oracle.fmm(np.ones((n, n)), h, [m * n + m]).t
        y, x = np.mgrid[0:n, 0:n]
        exact = np.hypot(x - m, y - m) * h
        errs.append(np.max(np.abs(t - exact)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.05


def test_unreachable_stays_inf():
    # a source time of +inf is not a source of anything; a 1-cell grid keeps t0
    t = oracle.fmm(np.ones((1, 1)), 1.0, [0], [0.25]).t
    assert t[0, 0] == 0.25


def test_duplicate_sources_take_the_min():
    t = oracle.fmm(np.ones((5, 5)), 1.0, [12, 12], [0.5, 0.25]).t
    assert t[2, 2] == 0.25


@pytest.mark.slow
def test_const_2d_129_matches_brute_force_sweeps():
    p = synth.const_2d_129()
    f = oracle.fmm(p.speed, p.h, p.sources)
    s = oracle.sweep(p.speed, p.h, p.sources, mode=1)
    assert np.array_equal(f.t, s.t)
    assert np.array_equal(f.t, f.t.T) and np.array_equal(f.t, f.t[::-1, ::-1])
    assert oracle.residual(p.speed, p.h, p.sources, f.t) == (0, 0.0)

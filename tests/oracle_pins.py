"""Reference facts the oracle is pinned to, independent of its code.

Each helper here computes something the paper or plain mathematics fixes:
exact real roots in 80-digit decimal arithmetic, the printed table values, and
closed-form arrival times.  The mutation test reuses these checks against
deliberately broken copies of the oracle.
"""
from __future__ import annotations

import math
import os
from decimal import Decimal, getcontext

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INF = float("inf")


def read_table(name: str):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            case, *vals = line.split()
            rows.append((case, *[float(v) for v in vals]))
    return rows


def exact_root(a, c: float) -> Decimal:
    """Real root of sum_k max(tau - a_k, 0)^2 = c (no rounding anywhere), the
    equation behind Eq. finite_difference with the max(., 0) upwind terms,
    solved with 80 significant digits.  +inf if every a_k is +inf."""
    getcontext().prec = 80
    b = sorted(Decimal(x) for x in a if x != INF)
    if not b:
        return Decimal("Infinity")
    C = Decimal(c)
    for j in range(1, len(b) + 1):
        S = sum(b[:j])
        Q = sum(x * x for x in b[:j])
        disc = S * S - j * (Q - C)
        tau = (S + disc.sqrt()) / j
        if j == len(b) or tau <= b[j]:
            return tau
    raise AssertionError("unreachable")


def ulps_from(x: float, ref: Decimal) -> float:
    """|x - ref| in units of ulp(x)."""
    return float(abs(Decimal(x) - ref) / Decimal(math.ulp(x)))


def random_minima(rng: np.random.Generator, D: int):
    """Axis minima near a large arrival time with random spreads, some +inf."""
    base = float(rng.uniform(0.0, 5000.0)) * float(rng.choice([1e-6, 1e-3, 1.0]))
    r = float(rng.uniform(0.01, 2.0)) * max(base, 1e-3) * float(rng.choice([1e-4, 1e-2, 0.3]))
    a = [base + float(rng.uniform(0.0, 1.5)) * r for _ in range(D)]
    for k in range(D):
        if rng.random() < 0.2:
            a[k] = INF
    if all(x == INF for x in a):
        a[int(rng.integers(D))] = base
    return a, r


def check_dbar_against_exact_root(dbar_fn, n: int = 400, seed: int = 11, tol_ulps: float = 4.0):
    """d-bar lies within a few ulps of the exact real root (rounding of G moves
    the threshold by at most ~3 ulps of tau).  Returns the worst distance."""
    rng = np.random.Generator(np.random.PCG64(seed))
    worst = 0.0
    for i in range(n):
        D = 2 if i % 2 == 0 else 3
        a, r = random_minima(rng, D)
        c = r * r
        d = dbar_fn(a, r, c)
        ref = exact_root(a, c)
        u = ulps_from(d, ref)
        worst = max(worst, u)
        if u > tol_ulps:
            raise AssertionError(f"dbar({a}, r={r!r}) = {d!r} is {u} ulps from the exact root {ref}")
    return worst


def closed_form_axis(n: int = 33, h: float = 2.0 ** -7):
    """Constant speed 1, dyadic h, point source at the centre of an n x n grid:
    arrival time along the axes through the source is exactly |k| h."""
    speed = np.ones((n, n))
    m = n // 2
    return speed, h, [m * n + m], m


def g_xyz(tau: float, a) -> float:
    """G(tau) of the definition in Python floats (IEEE binary64, one rounding per
    operation, no fused multiply-add): m_k = max(tau - a_k, 0), terms added in
    axis order x, y, z starting from the x term."""
    g = None
    for ak in a:
        m = tau - ak
        if not m > 0.0:
            m = 0.0
        q = m * m
        g = q if g is None else g + q
    return g


def certified_dbar(tau: float, a, c: float) -> bool:
    """tau is the smallest double with G(tau) >= c (the definition of d-bar)."""
    return g_xyz(tau, a) >= c and g_xyz(math.nextafter(tau, -math.inf), a) < c


def fixed_point_violations(speed: np.ndarray, h: float, sources, t: np.ndarray) -> int:
    """Cells of a solved grid where t is not d-bar of its neighbours' values, with
    c = fl(fl(h / v)^2) and G in x, y, z order, all in Python floats (sources:
    their time must be finite and unchanged by the check)."""
    src = set(int(s) for s in np.atleast_1d(sources))
    tt = np.asarray(t, dtype=np.float64)
    shape = tt.shape
    flat = tt.reshape(-1)
    bad = 0
    for idx in range(flat.size):
        if idx in src:
            continue
        coord = np.unravel_index(idx, shape)
        a = []
        for ax in range(len(shape) - 1, -1, -1):      # x (last axis) first
            best = math.inf
            for step in (-1, 1):
                cc = list(coord)
                cc[ax] += step
                if 0 <= cc[ax] < shape[ax]:
                    best = min(best, float(tt[tuple(cc)]))
            a.append(best)
        r = h / float(speed[coord])
        c = r * r
        ti = float(flat[idx])
        if all(x == math.inf for x in a):
            bad += ti != math.inf
        elif not certified_dbar(ti, a, c):
            bad += 1
    return bad


def run_pin_suite(orc) -> list[str]:
    """Run the cheap pins against an oracle module; return the names that fail."""
    import synth
    failed = []

    def pin(name, fn):
        try:
            ok = fn()
        except Exception:  # a crash or a wrong shape is a failed pin
            ok = False
        if not ok:
            failed.append(name)

    def tables():
        for table, fn in (("table1_dtilde.txt", orc.dtilde), ("table2_dhat.txt", orc.dhat)):
            for _, v, h, tH, tV, expect in read_table(table):
                if fn(v, h, tH, tV) != expect:
                    return False
        return True

    def roots():
        check_dbar_against_exact_root(lambda a, r, c: orc.dbar(a, r, c), n=150, seed=3)
        return True

    def axes():
        speed, h, src, m = closed_form_axis(17)
        t = orc.fmm(speed, h, src).t
        return all(t[m, m + k] == abs(k) * h and t[m + k, m] == abs(k) * h
                   for k in range(-m, m + 1))

    def plane3d():
        shape = (5, 6, 7)
        h = 2.0 ** -6
        idx = np.arange(np.prod(shape)).reshape(shape)
        t = orc.fmm(np.ones(shape), h, idx[:, :, 0].ravel()).t
        return np.array_equal(t, np.broadcast_to(np.arange(7) * h, shape))

    def line():
        rng = np.random.Generator(np.random.PCG64(21))
        speed = rng.uniform(1.0, 10.0, (1, 25))
        t = orc.fmm(speed, 0.37, [0]).t.ravel()
        return all(ulps_from(t[k], exact_root([t[k - 1]], (0.37 / speed[0, k]) ** 2)) <= 2.0
                   for k in range(1, t.size))

    def schedules():
        for shape in ((7, 9), (4, 5, 6)):
            p = synth.random_problem(3, shape, n_src=2, contrast=10.0, h=0.25)
            f = orc.fmm(p.speed, p.h, p.sources).t
            s = orc.sweep(p.speed, p.h, p.sources, mode=1).t
            if not np.array_equal(f, s):
                return False
            if orc.residual(p.speed, p.h, p.sources, f) != (0, 0.0):
                return False
        return True

    def dbar_definition():
        # d-bar against its definition in Python floats: random 2D / 3D minima in
        # axis order (not sorted), c = fl(fl(h / v)^2) from non-dyadic h and v
        rng = np.random.Generator(np.random.PCG64(29))
        for i in range(3000):
            D = 2 if i % 3 == 0 else 3
            a, _ = random_minima(rng, D)
            h = float(rng.uniform(0.1, 20.0))
            base = min(x for x in a if x != INF)
            v = h / (float(rng.uniform(0.05, 1.0)) * max(base, 1e-3) * float(rng.choice([1e-3, 0.05, 0.5])))
            r = h / v
            if not certified_dbar(orc.dbar(a, r, r * r), a, r * r):
                return False
        return True

    def grid_definition():
        # every cell of small solved grids (2D and 3D, non-dyadic spacing, 10:1
        # speeds) is d-bar of its neighbours by the Python-float definition
        for shape, seed in (((1, 40), 5), ((9, 11), 6), ((5, 6, 7), 7)):
            p = synth.random_problem(seed, shape, n_src=2, contrast=10.0, h=0.37)
            t = orc.fmm(p.speed, p.h, p.sources).t
            if fixed_point_violations(p.speed, p.h, p.sources, t):
                return False
        return True

    pin("tables", tables)
    pin("dbar_definition", dbar_definition)
    pin("grid_definition", grid_definition)
    pin("exact_roots", roots)
    pin("axes", axes)
    pin("plane3d", plane3d)
    pin("line", line)
    pin("schedules", schedules)
    return failed

"""Pins of the oracle adjoint (d loss / d slowness through the fixed point) to
central finite differences of the oracle forward solve and to the 1D closed
form d t_k / d s_j = h (j <= k)."""
import numpy as np
import pytest

import oracle
import synth


def test_line_closed_form():
    rng = np.random.Generator(np.random.PCG64(1))
    speed = rng.uniform(1.0, 3.0, (1, 40))
    h = 0.5
    t = oracle.fmm(speed, h, [0]).t
    g = np.zeros_like(t)
    g[0, -1] = 1.0
    g[0, 20] = 2.0
    _, gs = oracle.adjoint(speed, h, [0], t, g)
    expect = np.zeros(40)
    expect[1:21] = 3.0 * h
    expect[21:] = 1.0 * h
    assert gs[0, 0] == 0.0
    assert np.allclose(gs[0], expect, rtol=1e-12, atol=0)


def _fd_check(p, rcv_mask, cells, rel=1e-6):
    t = oracle.fmm(p.speed, p.h, p.sources).t
    target = t * 1.02 + 0.001
    g = np.where(rcv_mask, t - target, 0.0)
    _, gs = oracle.adjoint(p.speed, p.h, p.sources, t, g)
    s = 1.0 / p.speed

    def loss(speed):
        tt = oracle.fmm(speed, p.h, p.sources).t
        return 0.5 * np.sum(np.where(rcv_mask, tt - target, 0.0) ** 2)

    fds = []
    for j in cells:
        eps = 1e-7 * s[j]
        sp1 = p.speed.copy()
        sp1[j] = 1.0 / (s[j] + eps)
        sp2 = p.speed.copy()
        sp2[j] = 1.0 / (s[j] - eps)
        fds.append((loss(sp1) - loss(sp2)) / (2.0 * eps))
    fds = np.array(fds)
    ad = np.array([gs[j] for j in cells])
    scale = np.maximum(np.abs(fds), 1e-3 * np.abs(fds).max())
    return fds, ad, scale


@pytest.mark.parametrize("shape,seed", [((14, 17), 2), ((9, 10, 11), 3)])
def test_adjoint_matches_central_differences(shape, seed):
    p = synth.random_problem(seed, shape, n_src=2, contrast=4.0, smooth_sigma=1.5, h=1.0)
    rcv = np.zeros(shape, bool)
    rcv[(0,) * (len(shape) - 1)] = True        # a receiver line along x at the grid edge
    rcv.reshape(-1)[::7] = True
    rng = np.random.Generator(np.random.PCG64(seed))
    cells = [tuple(rng.integers(0, n) for n in shape) for _ in range(40)]
    fds, ad, scale = _fd_check(p, rcv, cells)
    assert np.abs(fds).max() > 0
    err = np.abs(ad - fds) / scale
    assert np.all(err < 1e-6), err.max()


def test_tomography_shaped_gradient_fourth_order_differences():
    """The 1024^2 tomography layout cut to 256^2 (surface sources and receivers,
    anomalies in the illuminated depth): the oracle gradient of
    L = 1/2 sum (t - t_obs)^2 against the fourth-order central stencil
    (8 D(eps) - D(2 eps)) / (12 eps), D(e) = L(s + e) - L(s - e), eps = 1e-4 s."""
    cfg = synth.tomography_2d_1024(n=256, n_src=2, n_rcv=128)
    h, rcv = cfg["h"], cfg["receivers"]
    s0 = 1.0 / cfg["start"]
    v = 1.0 / s0
    srcs = [[int(i)] for i in cfg["sources"]]
    t_obs = [oracle.fmm(cfg["true"], h, sv).t.reshape(-1)[rcv] for sv in srcs]
    grad = np.zeros(v.shape)
    for sv, to in zip(srcs, t_obs):
        t = oracle.fmm(v, h, sv).t
        g = np.zeros(v.shape)
        g.reshape(-1)[rcv] = t.reshape(-1)[rcv] - to
        assert np.abs(g).max() > 1e-4          # the anomalies are seen at the receivers
        grad += oracle.adjoint(v, h, sv, t, g)[1]
    flat = grad.reshape(-1)
    gmax = np.abs(flat).max()
    cand = np.nonzero(np.abs(flat) > 1e-6 * gmax)[0]
    cells = np.random.Generator(np.random.PCG64(7)).choice(cand, size=8, replace=False)

    def D(c, e):
        out = 0.0
        for sv, to in zip(srcs, t_obs):
            sp = s0.copy().reshape(-1)
            sp[c] += e
            tp = oracle.fmm(1.0 / sp.reshape(v.shape), h, sv).t.reshape(-1)[rcv]
            sp = s0.copy().reshape(-1)
            sp[c] -= e
            tm = oracle.fmm(1.0 / sp.reshape(v.shape), h, sv).t.reshape(-1)[rcv]
            out += 0.5 * np.sum((tp - tm) * (tp + tm - 2.0 * to))
        return out

    for c in cells:
        eps = 1e-4 * s0.reshape(-1)[c]
        fd = (8.0 * D(c, eps) - D(c, 2.0 * eps)) / (12.0 * eps)
        assert abs(flat[c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * gmax), (c, fd, flat[c])

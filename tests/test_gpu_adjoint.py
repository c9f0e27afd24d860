"""The GPU adjoint (eik_adjoint through the C ABI) equals the CPU oracle adjoint
bit for bit, and the tomography gradient of the differentiable batched solve
matches central finite differences (relative 1e-6) on the 1024^2 workload."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_05694_gb300 as eik  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2103_05694_gb300 import build
    build.build()
    eik.load_library()


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


SCHEDULES = {"levels": eik.ADJ_LEVELS, "tiles": eik.ADJ_TILES}


@pytest.mark.parametrize("sched", sorted(SCHEDULES))
@pytest.mark.parametrize("shape", [(40, 70), (3, 300), (12, 15, 17), (1, 1), (33, 1), (5, 9, 1),
                                   (17, 16, 9)])
def test_adjoint_bit_exact_vs_oracle(shape, sched):
    rng = np.random.Generator(np.random.PCG64(5))
    probs, ref = [], []
    base = synth.random_problem(21, shape, n_src=1, contrast=6.0, smooth_sigma=1.0, h=0.5)
    speed = torch.from_numpy(base.speed).to(DEV)
    for k in range(4):
        src = rng.choice(base.speed.size, size=min(1 + k % 3, base.speed.size),
                         replace=False).astype(np.int64)
        t = oracle.fmm(base.speed, base.h, src).t
        g = np.where(rng.random(shape) < 0.05, rng.standard_normal(shape), 0.0)
        lam, gs = oracle.adjoint(base.speed, base.h, src, t, g)
        ref.append(gs)
        out = torch.from_numpy(t).to(DEV)
        probs.append(dict(speed=speed, h=base.h, sources=torch.from_numpy(src).to(DEV), out=out,
                          g=torch.from_numpy(g).to(DEV), grad=torch.full_like(out, np.nan)))
    st = eik.eik_adjoint([{k: p[k] for k in ("speed", "h", "sources", "out")} for p in probs],
                         [p["g"] for p in probs], [p["grad"] for p in probs],
                         opts={"sched_flags": SCHEDULES[sched], "timeout_ms": 10000})
    torch.cuda.synchronize()
    for p, r in zip(probs, ref):
        got = p["grad"].cpu().numpy()
        assert np.array_equal(got.view(np.uint64), r.view(np.uint64))
    assert st["good"] == st["evals"] == sum(int(np.isfinite(p["out"].cpu().numpy()).sum())
                                            for p in probs)
    if sched == "tiles":
        assert st["visits"] >= 1 and st["ctas"] >= 1


def test_autograd_function_matches_oracle_adjoint():
    p = synth.random_problem(8, (30, 40), n_src=1, contrast=4.0, smooth_sigma=2.0, h=1.0)
    s = torch.from_numpy(1.0 / p.speed).to(DEV).requires_grad_(True)
    srcs = [torch.tensor([0], device=DEV), torch.tensor([39, 600], device=DEV)]
    t = eik.eikonal(s, p.h, srcs)
    w = torch.from_numpy(np.random.default_rng(0).random((2, 30, 40))).to(DEV)
    loss = 0.5 * (t * w).sum()
    loss.backward()
    speed = (1.0 / (1.0 / p.speed))      # the forward passes v = fl(1/s)
    v_used = 1.0 / s.detach().cpu().numpy()
    total = np.zeros((30, 40))
    for i, src in enumerate([[0], [39, 600]]):
        tt = oracle.fmm(v_used, p.h, src).t
        assert np.array_equal(tt, t[i].detach().cpu().numpy())
        _, gs = oracle.adjoint(v_used, p.h, src, tt, 0.5 * w[i].cpu().numpy())
        total = total + gs
    got = s.grad.cpu().numpy()
    # the library converts slowness on the device and sums the per-source
    # gradients from +0 in source order, as the loop above does
    assert np.array_equal(got.view(np.uint64), total.view(np.uint64))
    del speed


@pytest.mark.parametrize("sched", sorted(SCHEDULES))
def test_slowness_input_and_ordered_gradient_sum(sched):
    """sched_flags bit 6 (slowness in, v = fl(1/s) on the device) and bit 7
    (problems sharing a gradient array receive +0 + g_0 + g_1 + ... in problem
    order): equal to the oracle forward and adjoint run on v = 1/s and summed
    in the same order, bit for bit; two groups of outputs, one of them with a
    single problem."""
    rng = np.random.Generator(np.random.PCG64(77))
    shape = (23, 31) if sched == "levels" else (9, 11, 13)
    base = synth.random_problem(41, shape, n_src=1, contrast=5.0, smooth_sigma=1.0, h=0.75)
    s_np = 1.0 / base.speed
    v = 1.0 / s_np
    slow = torch.from_numpy(s_np).to(DEV)
    N = s_np.size
    srcs = [rng.choice(N, size=1 + k % 2, replace=False).astype(np.int64) for k in range(4)]
    outs = [torch.empty_like(slow) for _ in srcs]
    probs = [{"speed": slow, "h": base.h, "sources": torch.from_numpy(src).to(DEV), "out": o}
             for src, o in zip(srcs, outs)]
    eik.eik_solve_batched(probs, {"sched_flags": eik.SLOWNESS_INPUT})
    gs_dev = [torch.from_numpy(rng.standard_normal(shape) * (rng.random(shape) < 0.2)).to(DEV)
              for _ in srcs]
    shared, single = torch.full_like(slow, np.nan), torch.full_like(slow, np.nan)
    eik.eik_adjoint(probs, gs_dev, [shared, single, shared, shared],
                    {"sched_flags": eik.SLOWNESS_INPUT | eik.SUM_SHARED_GRADIENTS | SCHEDULES[sched],
                     "timeout_ms": 10000})
    torch.cuda.synchronize()
    want_shared, want_single = np.zeros(shape), np.zeros(shape)
    for k, (src, o, g) in enumerate(zip(srcs, outs, gs_dev)):
        t = oracle.fmm(v, base.h, src).t
        assert np.array_equal(o.cpu().numpy().view(np.uint64), t.view(np.uint64))
        gk = oracle.adjoint(v, base.h, src, t, g.cpu().numpy())[1]
        if k == 1:
            want_single = want_single + gk
        else:
            want_shared = want_shared + gk
    assert np.array_equal(shared.cpu().numpy().view(np.uint64), want_shared.view(np.uint64))
    assert np.array_equal(single.cpu().numpy().view(np.uint64), want_single.view(np.uint64))


@pytest.mark.parametrize("sched", sorted(SCHEDULES))
def test_adjoint_bit_exact_vs_oracle_tomography_grid(sched):
    """The 1024^2 tomography layout, two surface sources in one batch: forward
    times and the adjoint gradient both equal the oracle's bit for bit."""
    cfg = synth.tomography_2d_1024()
    h, rcv = cfg["h"], cfg["receivers"]
    v = 1.0 / (1.0 / cfg["start"])
    speed = torch.from_numpy(v).to(DEV)
    probs, ref = [], []
    for k in (0, 17):
        src = np.array([int(cfg["sources"][k])], dtype=np.int64)
        t = oracle.fmm(v, h, src).t
        t_obs = oracle.fmm(cfg["true"], h, src).t
        g = np.zeros(v.shape)
        g.reshape(-1)[rcv] = (t - t_obs).reshape(-1)[rcv]
        ref.append((t, oracle.adjoint(v, h, src, t, g)[1]))
        out = torch.empty_like(speed)
        probs.append(dict(speed=speed, h=h, sources=torch.from_numpy(src).to(DEV), out=out,
                          g=torch.from_numpy(g).to(DEV), grad=torch.full_like(out, np.nan)))
    eik.eik_solve_batched([{k: p[k] for k in ("speed", "h", "sources", "out")} for p in probs])
    eik.eik_adjoint([{k: p[k] for k in ("speed", "h", "sources", "out")} for p in probs],
                    [p["g"] for p in probs], [p["grad"] for p in probs],
                    opts={"sched_flags": SCHEDULES[sched], "timeout_ms": 10000})
    torch.cuda.synchronize()
    for p, (t, gs) in zip(probs, ref):
        assert np.array_equal(p["out"].cpu().numpy().view(np.uint64), t.view(np.uint64))
        assert np.array_equal(p["grad"].cpu().numpy().view(np.uint64), gs.view(np.uint64))


def _upwind_masks(t):
    """Per cell of a (sources, ny, nx) stack of fields: for each axis, which side
    holds the axis minimum (low, high or a tie) and whether the axis is active
    (minimum below the cell's time).  Two fields with equal masks everywhere
    are solutions of the same local equations (no upwind switch between them)."""
    inf = torch.full_like(t[..., :1], float("inf"))
    codes = []
    for ax in (2, 1):
        tt = t if ax == 2 else t.transpose(1, 2)
        lo = torch.cat([inf, tt[..., :-1]], dim=-1)
        hi = torch.cat([tt[..., 1:], inf], dim=-1)
        side = (lo < hi).to(torch.int8) + 2 * (hi < lo).to(torch.int8)     # 0 = tie
        active = (torch.minimum(lo, hi) < tt).to(torch.int8)
        code = side + 4 * active
        codes.append(code if ax == 2 else code.transpose(1, 2))
    return codes[0] + 8 * codes[1]


@pytest.mark.slow
def test_tomography_gradient_central_differences():
    """1024^2, 32 sources, 512 receivers, L = 1/2 sum (t - t_obs)^2.  Finite
    differences on 64 random cells (among those with |g| above 1e-6 of the
    largest) with the fourth-order central stencil
    (8 D(eps) - D(2 eps)) / (12 eps), D(e) = L(s + e) - L(s - e), eps = 1e-4 s.
    D is formed from t+ - t- so it does not cancel in L itself.  A step of
    1e-4 keeps the rounding of the perturbed times (a few ulps, ~1e-8 of the
    difference) and the stencil's eps^4 term far below the tolerance.
    Relative error against max(|g_FD|, 1e-3 max|g|) must be <= 1e-6, except at
    cells whose perturbations switch an upwind choice somewhere in the 32
    fields (the upwind masks of the four perturbed solutions differ: the loss
    has a kink inside the stencil, so central differences do not estimate the
    derivative there).  Those cells are listed; every other cell must pass.
    The four perturbed fields x 32 sources of one cell run as one batch."""
    cfg = synth.tomography_2d_1024()
    h = cfg["h"]
    n = cfg["start"].shape[0]
    s_true = torch.from_numpy(1.0 / cfg["true"]).to(DEV)
    s0 = torch.from_numpy(1.0 / cfg["start"]).to(DEV)
    srcs = [torch.tensor([int(i)], device=DEV) for i in cfg["sources"]]
    rcv = torch.from_numpy(cfg["receivers"]).to(DEV)
    with torch.no_grad():
        t_obs = eik.eikonal(s_true, h, srcs).reshape(len(srcs), -1)[:, rcv]
    assert float((t_obs > 0).float().mean()) == 1.0

    s = s0.clone().requires_grad_(True)
    L = 0.5 * ((eik.eikonal(s, h, srcs).reshape(len(srcs), -1)[:, rcv] - t_obs) ** 2).sum()
    L.backward()
    flat = s.grad.detach().reshape(-1)
    gmax = float(flat.abs().max())
    assert gmax > 0
    cand = torch.nonzero(flat.abs() > 1e-6 * gmax).reshape(-1).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(64))
    cells = rng.choice(cand, size=64, replace=False)

    steps = (1.0, -1.0, 2.0, -2.0)          # multiples of eps
    speeds = [torch.empty_like(s0) for _ in steps]
    outs = [torch.empty((len(srcs), n, n), dtype=torch.float64, device=DEV) for _ in steps]
    probs = [{"speed": speeds[j], "h": h, "sources": src, "out": outs[j][i]}
             for j in range(len(steps)) for i, src in enumerate(srcs)]
    fd, kink = [], []
    with torch.no_grad():
        for c in cells:
            eps = 1e-4 * float(s0.reshape(-1)[c])
            for j, m in enumerate(steps):
                sp = s0.clone().reshape(-1)
                sp[c] += m * eps
                speeds[j].copy_(sp.reshape(n, n))
            eik.eik_solve_batched(probs, {"sched_flags": eik.SLOWNESS_INPUT})
            tr = [outs[j].reshape(len(srcs), -1)[:, rcv] for j in range(len(steps))]
            masks = [_upwind_masks(outs[j]) for j in range(len(steps))]
            kink.append(any(not torch.equal(masks[0], mk) for mk in masks[1:]))

            def D(jp, jm):
                return float(0.5 * ((tr[jp] - tr[jm]) * (tr[jp] + tr[jm] - 2.0 * t_obs)).sum())
            fd.append((8.0 * D(0, 1) - D(2, 3)) / (12.0 * eps))
    fd = np.array(fd)
    kink = np.array(kink)
    ad = flat[torch.from_numpy(cells).to(DEV)].cpu().numpy()
    scale = np.maximum(np.abs(fd), 1e-3 * gmax)
    err = np.abs(ad - fd) / scale
    over = err > 1e-6
    print("tomography FD: median rel err %.2e, max over smooth cells %.2e; cells above 1e-6: %d "
          "(all at an upwind switch: cells %s, errors %s); upwind switches at %d cells"
          % (np.median(err), err[~kink].max() if (~kink).any() else 0.0, int(over.sum()),
             cells[over].tolist(), np.round(err[over], 9).tolist(), int(kink.sum())))
    assert np.median(err) <= 1e-6, (np.median(err), err.max())
    unexplained = over & ~kink
    assert not unexplained.any(), (cells[unexplained], err[unexplained])


def test_sum_ordered_bits():
    """eik_sum_ordered: +0 + x_0 + x_1 + ... in list order, each addition
    rounded to nearest, bit for bit as a sequential sum on the host; the order
    matters for these inputs; k = 0 writes +0."""
    rng = np.random.Generator(np.random.PCG64(12))
    xs = [rng.standard_normal(50_001) * 10.0 ** rng.integers(-12, 12, 50_001) for _ in range(9)]
    dev = [torch.from_numpy(x).to(DEV) for x in xs]
    out = torch.full_like(dev[0], np.nan)
    eik.eik_sum_ordered(dev, out)
    want = np.zeros(xs[0].shape)
    for x in xs:
        want = want + x
    assert np.array_equal(_bits(out.cpu().numpy()), _bits(want))
    rev = np.zeros(xs[0].shape)
    for x in xs[::-1]:
        rev = rev + x
    assert not np.array_equal(_bits(rev), _bits(want))
    eik.eik_sum_ordered([], out)
    assert np.array_equal(_bits(out.cpu().numpy()), _bits(np.zeros(xs[0].shape)))

"""The update-form ablation through the C ABI: the device evaluation of
Algorithm 1 with d-tilde / d-hat / d-hat then Newton (and of d-bar) equals the
oracle bit for bit
and reproduces Tables 1 and 2; the device Table 3 residual equals the oracle's;
solves with the explicit forms stay within rounding of the exact field and are
not fixed points in general, while d-bar's residual is exactly 0."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_05694_gb300 as eik  # noqa: E402

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2103_05694_gb300 import build
    build.build()
    eik.load_library()


def _t(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device=DEV)


def _rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out.append(tuple(map(float, f[1:])))
    return np.array(out)


@pytest.mark.parametrize("form,table", [(1, "table1_dtilde.txt"), (2, "table2_dhat.txt")])
def test_device_update_reproduces_tables(form, table):
    rows = _rows(table)
    v, h, tH, tV, want = rows.T
    assert np.all(h == h[0])
    got = eik.eik_eval_update(form, _t(v), h[0], _t(tH), _t(tV)).cpu().numpy()
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("form", [0, 1, 2, 3])
def test_device_update_equals_oracle(form):
    rng = np.random.Generator(np.random.PCG64(40 + form))
    n = 4000
    h = 1.25
    v = rng.uniform(1500.0, 4500.0, n)
    r = h / v
    tH = rng.uniform(0.0, 3.0, n)
    tV = tH + rng.uniform(-1.5, 1.5, n) * r
    tV[::17] = np.inf
    tH[::23] = np.inf
    tV = np.abs(tV)
    got = eik.eik_eval_update(form, _t(v), h, _t(tH), _t(tV)).cpu().numpy()
    want = np.array([oracle.update_form(form, v[i], h, tH[i], tV[i]) for i in range(n)])
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def _gpu_field(p, opts):
    speed = torch.from_numpy(p.speed).to(DEV)
    src = torch.from_numpy(p.sources).to(DEV)
    out = torch.empty_like(speed)
    eik.solve(speed, p.h, src, out=out, opts=opts)
    torch.cuda.synchronize()
    return {"speed": speed, "h": p.h, "sources": src, "out": out}


@pytest.mark.parametrize("shape", [(60, 80), (9, 300)])
def test_device_residual_equals_oracle(shape):
    p = synth.random_problem(12, shape, n_src=2, contrast=6.0, smooth_sigma=2.0, h=0.5)
    for upd in (0, 1, 2, 3):
        prob = _gpu_field(p, {"update": upd})
        t = prob["out"].cpu().numpy()
        for form in (0, 1, 2, 3):
            got = eik.eik_residual(prob, form)
            want = oracle.residual(p.speed, p.h, p.sources, t, form=form)
            assert got == want, (upd, form, got, want)


@pytest.mark.parametrize("form", [1, 2])
def test_explicit_forms_stay_within_rounding_of_the_exact_field(form):
    p = synth.layered_2d_2301x751()
    exact = _gpu_field(p, {})
    assert eik.eik_residual(exact, 0) == (0, 0.0)          # Table 3: true monotonicity, 0
    approx = _gpu_field(p, {"update": form})
    a, e = approx["out"].cpu().numpy(), exact["out"].cpu().numpy()
    rel = np.max(np.abs(a - e) / np.maximum(e, 1e-300))
    assert rel < 1e-9
    n, worst = eik.eik_residual(approx, form)
    assert worst < 1e-9


def test_explicit_forms_rejected_where_undefined():
    speed3 = torch.ones((5, 6, 7), dtype=torch.float64, device=DEV)
    with pytest.raises(eik.EikError) as e:
        eik.solve(speed3, 1.0, [0], opts={"update": 1})
    assert e.value.status == eik.EIK_EINVAL
    speed2 = torch.ones((16, 16), dtype=torch.float64, device=DEV)
    probs = [{"speed": speed2, "h": 1.0, "sources": torch.tensor([0], device=DEV),
              "out": torch.empty_like(speed2)}]
    with pytest.raises(eik.EikError) as e:
        eik.eik_autotune(probs, base={"update": 2})
    assert e.value.status == eik.EIK_EINVAL
    with pytest.raises(eik.EikError) as e:
        eik.solve(speed2, 1.0, [0], opts={"update": 4})
    assert e.value.status == eik.EIK_EINVAL


def test_dbar_bits_do_not_depend_on_the_schedule():
    p = synth.random_problem(13, (300, 200), n_src=3, contrast=8.0, smooth_sigma=1.0, h=1.0)
    ref = None
    for opts in ({}, {"tile": 1}, {"tile": 2, "k_delta": 1}, {"k_delta": 64, "window": 1},
                 {"tile": 3, "band": 1}):
        t = _gpu_field(p, opts)["out"].cpu().numpy()
        if ref is None:
            ref = t
        assert np.array_equal(t.view(np.uint64), ref.view(np.uint64)), opts


@pytest.mark.parametrize("form", [1, 2, 3])
def test_change_tracking_solves_stay_within_rounding(form):
    """Change tracking (a recomputed value that differs, up or down, replaces the
    cell's value and re-activates its neighbours): the field stays within
    rounding of the exact one, and the device residual equals the oracle's."""
    p = synth.random_problem(14, (160, 230), n_src=2, contrast=8.0, smooth_sigma=1.5, h=0.5)
    exact = _gpu_field(p, {})["out"].cpu().numpy()
    prob = _gpu_field(p, {"update": form, "sched_flags": eik.TRACK_CHANGES})
    t = prob["out"].cpu().numpy()
    rel = np.max(np.abs(t - exact) / np.maximum(exact, 1e-300))
    assert rel < 1e-9, rel
    got = eik.eik_residual(prob, form)
    assert got == oracle.residual(p.speed, p.h, p.sources, t, form=form)


def test_change_tracking_needs_an_explicit_form():
    speed = torch.ones((16, 16), dtype=torch.float64, device=DEV)
    with pytest.raises(eik.EikError) as e:
        eik.solve(speed, 1.0, [0], opts={"sched_flags": eik.TRACK_CHANGES})
    assert e.value.status == eik.EIK_EINVAL

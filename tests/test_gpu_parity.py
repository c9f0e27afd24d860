"""Parity of the CUDA path (through the C ABI) with the CPU oracle: bit-exact FP64.

The fixed point of the exactly monotone update is unique (Theorem 1), so any
nonzero-ulp difference from the oracle's fast marching result is a bug.
Covers ragged tiles, 1-cell and 1-row grids, multiple and duplicate sources,
non-zero source times, both pointer kinds, the capacity-retry path, several
bucket widths, the full-size 2D and 3D workloads, and error statuses.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2103_05694_gb300 as eik  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2103_05694_gb300 import build
    build.build()
    eik.load_library()
    yield


DEV = "cuda:0"


def gpu_solve(p, opts=None, host=False):
    if host:
        out = np.empty(p.speed.shape)
        r = eik.solve(p.speed, p.h, p.sources, p.src_t, out=out, opts=opts)
        return out, r.stats
    speed = torch.from_numpy(np.ascontiguousarray(p.speed)).to(DEV)
    src = torch.from_numpy(p.sources).to(DEV)
    st = torch.from_numpy(np.asarray(p.src_t, np.float64)).to(DEV)
    r = eik.solve(speed, p.h, src, st, opts=opts)
    torch.cuda.synchronize()
    return r.t.cpu().numpy(), r.stats


def assert_bits_equal(got, ref, what=""):
    g = got.view(np.uint64)
    e = ref.view(np.uint64)
    if not np.array_equal(g, e):
        diff = np.argwhere(g != e)
        i = tuple(diff[0])
        raise AssertionError(f"{what}: {len(diff)} cells differ; first {i}: "
                             f"gpu {got[i]!r} oracle {ref[i]!r}")


SHAPES = [(1, 1), (1, 40), (40, 1), (8, 32), (9, 33), (17, 65), (100, 37), (64, 64),
          (3, 300), (300, 3),
          (1, 1, 1), (4, 4, 16), (5, 5, 5), (17, 5, 9), (9, 33, 5), (20, 21, 22), (2, 40, 3)]


ARITHS = [1, 2]    # d-bar on the FP64 unit / exact emulation on the integer pipes


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("seed", [0, 1])
def test_random_grids_bit_exact(shape, seed, arith):
    p = synth.random_problem(1000 + seed, shape, n_src=1 + 2 * seed, contrast=10.0,
                             src_t_max=0.3 * seed, h=0.5)
    ref = oracle.fmm(p.speed, p.h, p.sources, p.src_t).t
    got, _ = gpu_solve(p, opts={"arith": arith})
    assert_bits_equal(got, ref, f"{shape} seed {seed} arith {arith}")


@pytest.mark.parametrize("shape", [(200, 300), (40, 50, 60)])
def test_smooth_media_bit_exact(shape):
    p = synth.random_problem(77, shape, n_src=4, contrast=5.0, smooth_sigma=3.0, h=2.0)
    ref = oracle.fmm(p.speed, p.h, p.sources, p.src_t).t
    got, st = gpu_solve(p, opts={"counters": 1})
    assert_bits_equal(got, ref, str(shape))
    assert st["good"] == int(np.isfinite(ref).sum()) - len(np.unique(p.sources))
    assert st["evals"] >= st["decreases"] >= st["good"] > 0


def test_const_2d_129_bit_exact_and_closed_form():
    p = synth.const_2d_129()
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    got, _ = gpu_solve(p)
    assert_bits_equal(got, ref, "const_2d_129")
    m = 64
    for k in range(-m, m + 1):
        assert got[m, m + k] == abs(k) * p.h and got[m + k, m] == abs(k) * p.h


@pytest.mark.parametrize("arith", ARITHS)
def test_layered_2d_bit_exact(arith):
    p = synth.layered_2d_2301x751()
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    got, st = gpu_solve(p, opts={"counters": 1, "arith": arith})
    assert_bits_equal(got, ref, "layered_2d_2301x751")
    assert st["good"] == p.ncells - 1


_C3 = {}


def _checker_3d_ref():
    if not _C3:
        p = synth.checker_3d_256()
        _C3["p"] = p
        _C3["ref"] = oracle.fmm(p.speed, p.h, p.sources).t
    return _C3["p"], _C3["ref"]


@pytest.mark.slow
@pytest.mark.parametrize("arith", ARITHS)
def test_checker_3d_bit_exact(arith):
    p, ref = _checker_3d_ref()
    got, st = gpu_solve(p, opts={"counters": 1, "arith": arith})
    assert_bits_equal(got, ref, "checker_3d_256")
    assert st["good"] == p.ncells - 1


def test_host_and_device_pointers_agree():
    p = synth.random_problem(5, (70, 90), n_src=3, contrast=8.0)
    a, _ = gpu_solve(p)
    b, _ = gpu_solve(p, host=True)
    assert_bits_equal(a, b, "host vs device buffers")


def test_repeat_runs_identical():
    p = synth.random_problem(6, (180, 260), n_src=5, contrast=10.0, smooth_sigma=2.0)
    first, _ = gpu_solve(p)
    for _ in range(5):
        again, _ = gpu_solve(p)
        assert_bits_equal(again, first, "repeat")


@pytest.mark.parametrize("k_delta", [0.5, 4.0, 64.0, 4096.0])
def test_bucket_width_does_not_change_bits(k_delta):
    p = synth.random_problem(9, (90, 120), n_src=2, contrast=10.0)
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    got, _ = gpu_solve(p, opts={"k_delta": k_delta})
    assert_bits_equal(got, ref, f"k_delta {k_delta}")


def test_capacity_retry_is_exact():
    p = synth.random_problem(10, (256, 512), n_src=40, contrast=10.0)
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    got, st = gpu_solve(p, opts={"capacity": 16, "k_delta": 1e6, "counters": 1})
    assert_bits_equal(got, ref, "capacity retry")
    assert st["retries"] >= 1


def test_no_sources_all_inf():
    speed = torch.ones((10, 12), dtype=torch.float64, device=DEV)
    r = eik.solve(speed, 1.0, torch.empty(0, dtype=torch.int64, device=DEV))
    assert torch.isinf(r.t).all()


def test_duplicate_sources_take_min():
    speed = torch.ones((6, 7), dtype=torch.float64, device=DEV)
    r = eik.solve(speed, 1.0, [8, 8, 30], src_t=[0.5, 0.25, 0.0])
    t = r.t.cpu().numpy()
    ref = oracle.fmm(np.ones((6, 7)), 1.0, [8, 8, 30], [0.5, 0.25, 0.0]).t
    assert_bits_equal(t, ref, "duplicates")
    assert t.ravel()[8] == 0.25


@pytest.mark.parametrize("bad", ["zero", "negative", "nan", "inf"])
def test_bad_speed_is_einval(bad):
    v = np.ones((20, 20))
    v[7, 3] = {"zero": 0.0, "negative": -1.0, "nan": np.nan, "inf": np.inf}[bad]
    with pytest.raises(eik.EikError) as ei:
        eik.solve(torch.from_numpy(v).to(DEV), 1.0, [0])
    assert ei.value.status == eik.EIK_EINVAL
    # the context stays usable
    r = eik.solve(torch.ones((20, 20), dtype=torch.float64, device=DEV), 1.0, [0])
    assert r.t[0, 5].item() == 5.0


def test_bad_host_arguments_are_einval():
    speed = torch.ones((4, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(eik.EikError) as ei:
        eik.solve(speed, -1.0, [0])
    assert ei.value.status == eik.EIK_EINVAL
    with pytest.raises(eik.EikError):
        eik.solve(speed, 1.0, [16])
    with pytest.raises(eik.EikError):
        eik.solve(speed, 1.0, [0], src_t=[-0.5])


def test_bounded_wait_returns_timeout_and_context_survives():
    """A device wait on a flag nothing sets ends with EIK_ETIMEOUT (no trap);
    the next solve on the same context is exact."""
    p = synth.random_problem(11, (40, 50), n_src=1)
    with pytest.raises(eik.EikError) as ei:
        gpu_solve(p, opts={"test_stall": 1, "timeout_ms": 200})
    assert ei.value.status == eik.EIK_ETIMEOUT
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    got, _ = gpu_solve(p)
    assert_bits_equal(got, ref, "after timeout")

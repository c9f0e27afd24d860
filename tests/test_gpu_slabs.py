"""Slab decomposition of one grid (eik_solve_slabs): the outermost axis split
into K slabs solved by epochs with a one-row halo exchange gives the oracle's
fixed point bit for bit, for every K from 1 to one row per slab, with sources
inside slabs, on slab boundaries and with non-zero source times; and on the
layered 2D section and the 3D checkerboard volume at full size."""
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


def _check(p, ks):
    ref = oracle.fmm(p.speed, p.h, p.sources, p.src_t).t
    speed = torch.from_numpy(p.speed).to(DEV)
    for k in ks:
        r = eik.solve_slabs(speed, p.h, p.sources, k, src_t=p.src_t, opts={"counters": 1})
        torch.cuda.synchronize()
        got = r.t.cpu().numpy()
        assert np.array_equal(_bits(got), _bits(ref)), (p.name, k, int(np.sum(got != ref)))
        assert r.stats["epochs"] >= 1
        assert r.stats["good"] == int(np.isfinite(ref).sum()) - len(np.unique(p.sources))


@pytest.mark.parametrize("shape,seed", [((23, 17), 1), ((9, 40), 2), ((12, 7, 9), 3), ((5, 6, 13), 4)])
def test_small_grids_every_slab_count(shape, seed):
    p = synth.random_problem(seed, shape, n_src=3, contrast=10.0, h=0.6, src_t_max=0.5)
    L = shape[0]
    _check(p, sorted({1, 2, 3, L // 2, L}))


def test_sources_on_slab_boundaries():
    # sources in the first and last row of slabs and in the rows next to them
    shape = (16, 21)
    rng = np.random.Generator(np.random.PCG64(9))
    speed = 1.0 + 9.0 * rng.random(shape)
    rows = [3, 4, 7, 8, 11, 12]
    src = np.array([r * shape[1] + int(rng.integers(shape[1])) for r in rows], dtype=np.int64)
    p = synth.Problem("boundary_sources", speed, 0.35, src, rng.random(len(rows)) * 0.1, {})
    _check(p, [2, 4, 5, 16])


def test_winding_path_needs_several_epochs():
    # a fast channel that leaves slab 0, runs through slab 1 and comes back:
    # cells of slab 0 are reached fastest through slab 1, so the exchange must
    # go back and forth
    ny, nx = 24, 60
    speed = np.full((ny, nx), 1.0)
    speed[14, :] = 50.0          # fast row in the lower half
    speed[2:15, 2] = 50.0        # down from the source row
    speed[2:15, nx - 3] = 50.0   # and back up at the far end
    p = synth.Problem("winding", speed, 1.0, np.array([2 * nx + 2], dtype=np.int64), np.zeros(1), {})
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    r = eik.solve_slabs(torch.from_numpy(speed).to(DEV), 1.0, p.sources, 2)
    torch.cuda.synchronize()
    assert np.array_equal(_bits(r.t.cpu().numpy()), _bits(ref))
    assert r.stats["epochs"] >= 3


def test_bad_arguments():
    speed = torch.ones((8, 8), dtype=torch.float64, device=DEV)
    for k in (0, 9):
        with pytest.raises(eik.EikError) as ei:
            eik.solve_slabs(speed, 1.0, [0], k)
        assert ei.value.status == eik.EIK_EINVAL
    with pytest.raises(eik.EikError):
        eik.solve_slabs(speed, 1.0, [0], 2, opts={"update": 2})


@pytest.mark.slow
def test_layered_section_full_size():
    _check(synth.layered_2d_2301x751(), [2, 4, 7])


@pytest.mark.slow
def test_checkerboard_volume_full_size():
    _check(synth.checker_3d_256(), [2, 4])

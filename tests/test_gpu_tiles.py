"""Every tile shape (opts.tile) reaches the oracle's fixed point bit for bit:
ragged edges, thin grids, several sources, batched problems and plans, and
the full-size 2D layered section.  Invalid shapes are EIK_EINVAL."""
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


def _bits_equal(got, ref, what):
    g, e = got.view(np.uint64), ref.view(np.uint64)
    assert np.array_equal(g, e), f"{what}: {int((g != e).sum())} cells differ"


SHAPES = [(1, 1), (7, 300), (33, 65), (100, 37), (64, 64), (300, 5),
          (1, 1, 1), (5, 5, 5), (17, 5, 9), (9, 33, 5), (20, 21, 22), (3, 40, 2)]


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("shape", SHAPES)
def test_tile_shapes_bit_exact(shape, tile):
    p = synth.random_problem(500 + len(shape) * 7 + shape[0], shape, n_src=3, contrast=8.0,
                             src_t_max=0.2, h=0.5)
    ref = oracle.fmm(p.speed, p.h, p.sources, p.src_t).t
    r = eik.solve(torch.from_numpy(p.speed).to(DEV), p.h, torch.from_numpy(p.sources).to(DEV),
                  torch.from_numpy(p.src_t).to(DEV), opts={"tile": tile, "counters": 1})
    torch.cuda.synchronize()
    _bits_equal(r.t.cpu().numpy(), ref, f"{shape} tile {tile}")
    assert r.stats["good"] == int(np.isfinite(ref).sum()) - len(np.unique(p.sources))


@pytest.mark.parametrize("tile", [2, 3, 4, 5])
def test_tile_shapes_layered_section(tile):
    p = synth.layered_2d_2301x751()
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    r = eik.solve(torch.from_numpy(p.speed).to(DEV), p.h, torch.from_numpy(p.sources).to(DEV),
                  opts={"tile": tile})
    torch.cuda.synchronize()
    _bits_equal(r.t.cpu().numpy(), ref, f"layered tile {tile}")


@pytest.mark.parametrize("tile", [0, 2, 4, 5])
def test_tile_shapes_batched_and_plan(tile):
    base = synth.random_problem(31, (30, 41, 23), n_src=1, contrast=6.0, smooth_sigma=1.5, h=1.0)
    speed = torch.from_numpy(base.speed).to(DEV)
    srcs = [np.array([5]), np.array([100, 2000]), np.array([base.speed.size - 1])]
    probs = [{"speed": speed, "h": base.h, "sources": torch.from_numpy(s).to(DEV),
              "out": torch.empty_like(speed)} for s in srcs]
    eik.eik_solve_batched(probs, {"tile": tile})
    plan = eik.Plan([{"speed": speed, "h": base.h, "sources": torch.from_numpy(s).to(DEV),
                      "out": torch.empty_like(speed)} for s in srcs], {"tile": tile})
    plan.enqueue()
    plan.status()
    torch.cuda.synchronize()
    for s, q, pq in zip(srcs, probs, plan.problems):
        ref = oracle.fmm(base.speed, base.h, s).t
        _bits_equal(q["out"].cpu().numpy(), ref, f"batched tile {tile}")
        _bits_equal(pq["out"].cpu().numpy(), ref, f"plan tile {tile}")
    plan.close()


@pytest.mark.parametrize("opts", [{"tile": 6}, {"tile": -1}, {"tile": 2, "arith": 2},
                                  {"tile": 6, "arith": 2}])
def test_bad_tile_is_einval(opts):
    speed = torch.ones((8, 9), dtype=torch.float64, device=DEV)
    with pytest.raises(eik.EikError) as e:
        eik.solve(speed, 1.0, [0], opts=opts)
    assert e.value.status == eik.EIK_EINVAL


def test_default_launch_configuration_3d():
    """3D defaults: 4x4x4 tiles; one front (under 8 sources) on 14 CTAs per SM,
    many fronts on the 20 of the wide lean build; a counting solve of many
    fronts on the 16 the counting build holds; the same bits as an explicit
    8x4x4 solve."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for n_src, per_sm in ((1, 14), (8, 20)):
        # 32,768 tiles: at least 8 per CTA, so no lane groups and the lean build
        p = synth.random_problem(900 + n_src, (128, 128, 128), n_src=n_src, contrast=6.0)
        speed = torch.from_numpy(np.ascontiguousarray(p.speed)).to(DEV)
        src = torch.from_numpy(p.sources).to(DEV)
        r = eik.solve(speed, p.h, src)
        assert r.stats["ctas"] == per_sm * sms, (n_src, r.stats["ctas"])
        r2 = eik.solve(speed, p.h, src, opts={"tile": 4})
        assert r2.stats["ctas"] == 8 * sms
        _bits_equal(r.t.cpu().numpy(), r2.t.cpu().numpy(), f"{n_src} sources")
        r3 = eik.solve(speed, p.h, src, opts={"counters": 1})
        assert r3.stats["ctas"] == min(per_sm, 16) * sms
        _bits_equal(r.t.cpu().numpy(), r3.t.cpu().numpy(), f"{n_src} sources, counting")
        # an explicit request above the normal build's 16 takes the wide build
        # (lean) or is capped at 16 (counting)
        r4 = eik.solve(speed, p.h, src, opts={"ctas_per_sm": 18})
        assert r4.stats["ctas"] == 18 * sms
        r5 = eik.solve(speed, p.h, src, opts={"ctas_per_sm": 18, "counters": 1})
        assert r5.stats["ctas"] == 16 * sms
        _bits_equal(r.t.cpu().numpy(), r4.t.cpu().numpy(), f"{n_src} sources, 18 CTAs per SM")
        _bits_equal(r.t.cpu().numpy(), r5.t.cpu().numpy(), f"{n_src} sources, 18 CTAs per SM, counting")

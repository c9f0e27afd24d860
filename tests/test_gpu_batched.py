"""Batched solves: many sources on a shared speed array plus grids of uneven
size, in one persistent launch (eik_solve_batched, and plans replayed from a
captured CUDA graph), bit-exact against the CPU oracle problem by problem."""
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


def _batch(ndim, seed=0):
    """Shared-model sources (one problem each) and independent uneven grids."""
    rng = np.random.Generator(np.random.PCG64(seed))
    probs = []
    if ndim == 3:
        model = synth.smooth_random_volume(24, 50 + seed, 1500.0, 4500.0, 3.0)
        h = 10.0
    else:
        model = synth.layered_section(120, 60, 4.0, seed=7 + seed)
        h = 4.0
    shared = torch.from_numpy(model).to(DEV)
    for k in range(6):
        src = int(rng.integers(0, model.size))
        probs.append(dict(name=f"shared{k}", np_speed=model, h=h, np_src=np.array([src]),
                          np_t=np.zeros(1), speed=shared))
    for k in range(5):
        if ndim == 3:
            side = int(rng.integers(7, 30))
            v = synth.smooth_random_volume(side, 90 + k + seed, 1500.0, 4500.0, 2.0)
        else:
            v = synth.random_problem(200 + k + seed, (int(rng.integers(5, 90)), int(rng.integers(5, 130))),
                                     contrast=8.0, smooth_sigma=1.0).speed
        ns = int(rng.integers(1, 5))
        src = rng.integers(0, v.size, ns)
        t0 = rng.random(ns) * 0.01
        probs.append(dict(name=f"grid{k}", np_speed=v, h=h, np_src=src, np_t=t0,
                          speed=torch.from_numpy(v).to(DEV)))
    for p in probs:
        p["sources"] = torch.from_numpy(np.asarray(p["np_src"], np.int64)).to(DEV)
        p["src_t"] = torch.from_numpy(np.asarray(p["np_t"], np.float64)).to(DEV)
        p["out"] = torch.full(p["np_speed"].shape, -1.0, dtype=torch.float64, device=DEV)
    return probs


def _check(probs):
    for p in probs:
        ref = oracle.fmm(p["np_speed"], p["h"], p["np_src"], p["np_t"]).t
        got = p["out"].cpu().numpy()
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), p["name"]


@pytest.mark.parametrize("ndim", [2, 3])
def test_solve_batched_bit_exact(ndim):
    probs = _batch(ndim)
    st = eik.eik_solve_batched([{k: p[k] for k in ("speed", "h", "sources", "src_t", "out")}
                                for p in probs], {"counters": 1})
    torch.cuda.synchronize()
    _check(probs)
    reached = sum(int(np.isfinite(p["out"].cpu().numpy()).sum()) - len(np.unique(p["np_src"]))
                  for p in probs)
    assert st["good"] == reached


@pytest.mark.parametrize("ndim", [2, 3])
def test_plan_graph_replay_bit_exact(ndim):
    probs = _batch(ndim, seed=1)
    plan = eik.Plan([{k: p[k] for k in ("speed", "h", "sources", "src_t", "out")} for p in probs],
                    {"counters": 1})
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan.enqueue(stream)          # warm-up solve outside the graph
    stream.synchronize()
    plan.status(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.enqueue(stream)
    for rep in range(3):
        for p in probs:
            p["out"].fill_(-1.0)
        g.replay()
        torch.cuda.synchronize()
        st = plan.status(torch.cuda.current_stream())
        _check(probs)
        assert st["good"] > 0
    plan.close()


@pytest.mark.parametrize("shape,k_delta", [((256, 384), 1.0), ((300, 200), 0.5), ((40, 48, 56), 0.5)])
def test_small_rings_and_narrow_buckets(shape, k_delta):
    """Rings of 16 entries per bucket slot (grown by the capacity retry when a
    bucket holds more) and buckets narrow enough that slots serve several
    buckets in turn: small, contended rings under the reservation protocol and
    the sequence-tagged positions still give the oracle's bits."""
    p = synth.random_problem(23, shape, n_src=1, contrast=6.0, smooth_sigma=1.5, h=1.0)
    r = eik.solve(torch.from_numpy(p.speed).to(DEV), p.h, torch.from_numpy(p.sources).to(DEV),
                  opts={"capacity": 16, "k_delta": k_delta, "counters": 1})
    torch.cuda.synchronize()
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    assert np.array_equal(r.t.cpu().numpy().view(np.uint64), ref.view(np.uint64))
    assert r.stats["pushes"] > 1000

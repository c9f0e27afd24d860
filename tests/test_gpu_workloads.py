"""The benchmark's batched workloads at full size, in the launch configuration
the benchmark times (the automatic tile shape and bucket width of a batch with
many wavefronts, one persistent launch for the whole batch): sampled problems
equal the CPU oracle bit for bit, forward and adjoint; every other problem
satisfies properties that hold at any size."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


def test_tomography_32_source_batch_sampled():
    """1024^2, 32 surface sources in one batch (16x8 tiles, k_delta 2: the bench's
    forward), then the tile-scheduled adjoint of the receiver misfit.  Three
    sources are checked against the oracle (times and gradient); every source's
    field is finite, non-negative and 0 at its source."""
    cfg = synth.tomography_2d_1024()
    h, rcv = cfg["h"], cfg["receivers"]
    v = 1.0 / (1.0 / cfg["start"])
    speed = torch.from_numpy(v).to(DEV)
    srcs = [int(s) for s in cfg["sources"]]
    probs = [{"speed": speed, "h": h, "sources": torch.tensor([s], device=DEV),
              "out": torch.empty_like(speed)} for s in srcs]
    eik.eik_solve_batched(probs)
    picks = (0, 13, 31)
    dl_dt = [torch.zeros_like(speed) for _ in srcs]
    refs = {}
    for k in picks:
        t = oracle.fmm(v, h, [srcs[k]]).t
        t_obs = oracle.fmm(cfg["true"], h, [srcs[k]]).t
        g = np.zeros(v.shape)
        g.reshape(-1)[rcv] = (t - t_obs).reshape(-1)[rcv]
        refs[k] = (t, oracle.adjoint(v, h, [srcs[k]], t, g)[1])
        dl_dt[k] = torch.from_numpy(g).to(DEV)
    grads = [torch.full_like(speed, np.nan) for _ in srcs]
    eik.eik_adjoint(probs, dl_dt, grads)
    torch.cuda.synchronize()
    for k in picks:
        t, gs = refs[k]
        assert np.array_equal(_bits(probs[k]["out"].cpu().numpy()), _bits(t)), k
        assert np.array_equal(_bits(grads[k].cpu().numpy()), _bits(gs)), k
    for k, p in enumerate(probs):
        t = p["out"].cpu().numpy()
        assert np.isfinite(t).all() and (t >= 0).all() and t.reshape(-1)[srcs[k]] == 0.0
        assert torch.count_nonzero(grads[k]).item() == 0 or k in picks   # zero misfit elsewhere


def test_batched_3d_full_batch_sampled():
    """The 88-problem 3D batch (64 sources on a shared 128^3 model, 24 uneven
    grids) as one plan, as the bench replays it.  Five problems are checked
    against the oracle; every field is finite, non-negative and t0 at its
    sources."""
    problems = synth.batched_3d()
    speeds = {}
    probs = []
    for p in problems:
        if id(p.speed) not in speeds:
            speeds[id(p.speed)] = torch.from_numpy(p.speed).to(DEV)
        sp = speeds[id(p.speed)]
        probs.append({"speed": sp, "h": p.h, "sources": torch.from_numpy(p.sources).to(DEV),
                      "out": torch.empty_like(sp)})
    plan = eik.Plan(probs)
    plan.enqueue()
    plan.status()
    torch.cuda.synchronize()
    grids = sorted(range(64, len(problems)), key=lambda i: problems[i].speed.size)
    for i in (0, 37, 63, grids[0], grids[1]):
        p = problems[i]
        ref = oracle.fmm(p.speed, p.h, p.sources, p.src_t).t
        assert np.array_equal(_bits(plan.problems[i]["out"].cpu().numpy()), _bits(ref)), p.name
    for p, q in zip(problems, plan.problems):
        t = q["out"].cpu().numpy()
        assert np.isfinite(t).all() and (t >= 0).all()
        assert np.all(t.reshape(-1)[p.sources] == p.src_t)
    plan.close()

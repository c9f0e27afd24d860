"""The autotuner (eik_autotune through the C ABI) tries configurations of the
scheduler, keeps the fastest, and every trial reproduces the same bits; the
chosen options give the oracle's fixed point."""
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


def _batch(shape, n, seed):
    base = synth.random_problem(seed, shape, n_src=1, contrast=5.0, smooth_sigma=2.0, h=1.0)
    speed = torch.from_numpy(base.speed).to(DEV)
    rng = np.random.Generator(np.random.PCG64(seed))
    srcs = [np.sort(rng.choice(base.speed.size, size=1 + k % 3, replace=False)) for k in range(n)]
    probs = [{"speed": speed, "h": base.h, "sources": torch.from_numpy(s.astype(np.int64)).to(DEV),
              "out": torch.empty_like(speed)} for s in srcs]
    return base, srcs, probs


@pytest.mark.parametrize("shape", [(160, 230), (40, 36, 44)])
def test_autotune_bits_and_choice(shape):
    base, srcs, probs = _batch(shape, 3, 11)
    best, trials = eik.eik_autotune(probs, repeats=1)
    assert len(trials) >= 10
    assert all(t["status"] == eik.EIK_OK and t["ms"] > 0 for t in trials)
    assert 1 <= best["tile"] <= 4 and best["k_delta"] > 0 and best["window"] > 0
    cap = best["capacity"]
    assert cap >= 64 and cap & (cap - 1) == 0
    # the chosen configuration is no slower than the starting one (same run)
    assert min(t["ms"] for t in trials) <= trials[0]["ms"]
    refs = [oracle.fmm(base.speed, base.h, s).t for s in srcs]
    for q, r in zip(probs, refs):          # outputs of the tuner's last solve
        assert np.array_equal(q["out"].cpu().numpy().view(np.uint64), r.view(np.uint64))
    for q in probs:
        q["out"].fill_(0.0)
    eik.eik_solve_batched(probs, best)
    torch.cuda.synchronize()
    for q, r in zip(probs, refs):
        assert np.array_equal(q["out"].cpu().numpy().view(np.uint64), r.view(np.uint64))


def test_autotune_respects_fixed_delta_and_capacity():
    _, _, probs = _batch((90, 70), 2, 12)
    best, trials = eik.eik_autotune(probs, base={"delta": 3.0, "capacity": 4096}, repeats=1)
    assert best["delta"] == 3.0 and best["capacity"] == 4096
    assert all(t["k_delta"] == trials[0]["k_delta"] for t in trials)


def test_autotune_rejects_host_pointers():
    speed = np.ones((8, 8))
    probs = [{"speed": speed, "h": 1.0, "sources": np.array([0], np.int64),
              "out": np.empty((8, 8))}]
    with pytest.raises(eik.EikError) as e:
        eik.eik_autotune(probs)
    assert e.value.status == eik.EIK_EINVAL

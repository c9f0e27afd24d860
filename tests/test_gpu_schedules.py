"""The comparison schedules of the same exact update (opts.schedule: the fast
iterative method, Algorithm 3 with epsilon = 0, the topology-driven schedule,
Algorithm 4, and the fast sweeping method, Algorithm 5) reach the oracle's
fixed point bit for bit (Theorem 1);
their work counters are consistent; misuse is EIK_EINVAL."""
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


def _solve(p, opts):
    speed = torch.from_numpy(p.speed).to(DEV)
    r = eik.solve(speed, p.h, torch.from_numpy(p.sources).to(DEV),
                  torch.from_numpy(np.asarray(p.src_t, np.float64)).to(DEV), opts=opts)
    torch.cuda.synchronize()
    return r.t.cpu().numpy(), r.stats


@pytest.mark.parametrize("schedule", [1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 1), (1, 50), (37, 45), (120, 90), (5, 5, 5), (17, 9, 23)])
def test_schedules_bit_exact(schedule, shape):
    p = synth.random_problem(900 + len(shape) + shape[-1], shape, n_src=2, contrast=8.0,
                             src_t_max=0.2, h=0.5)
    ref = oracle.fmm(p.speed, p.h, p.sources, p.src_t).t
    got, st = _solve(p, {"schedule": schedule, "counters": 1})
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    good = int(np.isfinite(ref).sum()) - len(np.unique(p.sources))
    assert st["good"] == good
    assert st["evals"] >= st["decreases"] >= good
    assert st["rounds"] >= 1


@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_schedules_on_the_layered_section_quarter(schedule):
    nx, nz = 575, 188
    speed = synth.layered_section(nx, nz, 4.0, seed=2)
    p = synth.Problem("layered_quarter", speed, 4.0, np.array([nx // 2], np.int64), np.zeros(1), {})
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    got, st = _solve(p, {"schedule": schedule, "counters": 1})
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    amm, st0 = _solve(p, {"counters": 1})
    assert np.array_equal(amm.view(np.uint64), got.view(np.uint64))
    assert st["good"] == st0["good"] == p.ncells - 1


def test_schedule_misuse_is_einval():
    speed = torch.ones((10, 12), dtype=torch.float64, device=DEV)
    for opts in ({"schedule": 4}, {"schedule": 1, "update": 1}, {"schedule": 2, "arith": 2}):
        with pytest.raises(eik.EikError) as e:
            eik.solve(speed, 1.0, [0], opts=opts)
        assert e.value.status == eik.EIK_EINVAL
    with pytest.raises(eik.EikError) as e:          # host pointers
        eik.solve(np.ones((10, 12)), 1.0, [0], opts={"schedule": 1})
    assert e.value.status == eik.EIK_EINVAL
    probs = [{"speed": speed, "h": 1.0, "sources": torch.tensor([0], device=DEV),
              "out": torch.empty_like(speed)} for _ in range(2)]
    with pytest.raises(eik.EikError) as e:          # batches
        eik.eik_solve_batched(probs, {"schedule": 1})
    assert e.value.status == eik.EIK_EINVAL

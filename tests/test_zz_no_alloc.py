"""eik_solve_noalloc, the solve that allocates no memory, gives the same bits
as eik_solve, on two calls in a row.

It exists for callers that cannot allocate device memory (their device memory
belongs to an arena allocator that forbids outside cudaMalloc calls, or their
loop cannot afford the device-wide synchronisation of cudaMalloc / cudaFree);
it runs the solver on a fixed scratch array instead.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

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


def _problems():
    p2 = synth.random_problem(31, (300, 400), n_src=5, contrast=10.0, src_t_max=0.2, h=0.5)
    # duplicate sources with different times: the smallest time must win
    src2 = np.concatenate([p2.sources, p2.sources[:2]])
    t2 = np.concatenate([p2.src_t, [0.0, p2.src_t[1] + 1.0]])
    p3 = synth.random_problem(32, (40, 50, 60), n_src=3, contrast=5.0, smooth_sigma=2.0, h=2.0)
    p1 = synth.const_2d_129()
    return [(p2.speed, p2.h, src2, t2), (p3.speed, p3.h, p3.sources, p3.src_t),
            (p1.speed, p1.h, p1.sources, None)]


@pytest.mark.parametrize("case", [0, 1, 2])
def test_noalloc_equals_eik_solve_twice(case):
    speed_np, h, src_np, t_np = _problems()[case]
    speed = torch.from_numpy(np.ascontiguousarray(speed_np)).to(DEV)
    src = torch.from_numpy(np.asarray(src_np, dtype=np.int64)).to(DEV)
    st = None if t_np is None else torch.from_numpy(np.asarray(t_np, np.float64)).to(DEV)
    ref = eik.solve(speed, h, src, st).t
    torch.cuda.synchronize()
    for _ in range(2):
        out = torch.full_like(speed, -1.0)
        stats = eik.eik_solve_noalloc(speed.data_ptr(), h, speed.ndim, speed.shape,
                                      src.data_ptr(), None if st is None else st.data_ptr(),
                                      src.numel(), out.data_ptr(), {"counters": 1},
                                      torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.int64), ref.view(torch.int64))
        assert stats["good"] == int(torch.isfinite(ref).sum().item()) - len(np.unique(src_np))


def test_noalloc_rejects_inputs_beyond_its_limits():
    big = torch.ones((1025, 1025), dtype=torch.float64, device=DEV)
    src = torch.zeros(1, dtype=torch.int64, device=DEV)
    out = torch.empty_like(big)
    with pytest.raises(eik.EikError) as ei:
        eik.eik_solve_noalloc(big.data_ptr(), 1.0, 2, big.shape, src.data_ptr(), None, 1,
                              out.data_ptr())
    assert ei.value.status == eik.EIK_EINVAL
    small = torch.ones((8, 8), dtype=torch.float64, device=DEV)
    out = torch.empty_like(small)
    many = torch.zeros(2049, dtype=torch.int64, device=DEV)
    with pytest.raises(eik.EikError):
        eik.eik_solve_noalloc(small.data_ptr(), 1.0, 2, small.shape, many.data_ptr(), None,
                              many.numel(), out.data_ptr())
    host = np.ones((8, 8))
    with pytest.raises(eik.EikError):
        eik.eik_solve_noalloc(host.ctypes.data, 1.0, 2, host.shape, src.data_ptr(), None, 1,
                              out.data_ptr())
    bad_src = torch.tensor([64], dtype=torch.int64, device=DEV)   # out of range: device check
    with pytest.raises(eik.EikError) as ei:
        eik.eik_solve_noalloc(small.data_ptr(), 1.0, 2, small.shape, bad_src.data_ptr(), None, 1,
                              out.data_ptr())
    assert ei.value.status == eik.EIK_EINVAL
    # the message names this call and the reason, not an earlier call's error
    assert "eik_solve_noalloc" in str(ei.value) and "sources" in str(ei.value)
    # still usable afterwards
    good = torch.zeros(1, dtype=torch.int64, device=DEV)
    eik.eik_solve_noalloc(small.data_ptr(), 1.0, 2, small.shape, good.data_ptr(), None, 1,
                          out.data_ptr())
    torch.cuda.synchronize()
    assert out[0, 7].item() == 7.0

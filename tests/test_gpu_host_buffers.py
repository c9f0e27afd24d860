"""Host buffers through the C ABI, bit for bit against the same problems on
device buffers and against the CPU oracle:

* pinned host memory (mapped into the device's address space) is read in
  place by the kernel that forms c and written by one copy kernel after the
  solve -- odd sizes (the copy kernel's 8-byte tail), an output that starts 8
  bytes into its allocation (no 16-byte accesses), a speed array shared by
  two problems;
* pageable host memory (numpy) takes the cudaMemcpyAsync path;
* a plan over pinned host buffers, enqueued twice (graph-capturable path);
* eik_solve on one pinned 3D grid."""
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


def _batch_2d():
    shapes = [(33, 47), (64, 65), (17, 19), (1, 1), (7, 129)]
    probs = [synth.random_problem(40 + i, s, n_src=1 + i % 3, contrast=6.0) for i, s in enumerate(shapes)]
    # the last problem reuses the first problem's speed array (shared speed)
    probs.append(synth.Problem(speed=probs[0].speed, h=probs[0].h,
                               sources=np.array([5, 700], dtype=np.int64),
                               src_t=np.zeros(2), name="shared"))
    return probs


def _device_reference(probs):
    dev = []
    for p in probs:
        sp = torch.from_numpy(np.ascontiguousarray(p.speed)).to(DEV)
        dev.append({"speed": sp, "h": p.h, "sources": torch.from_numpy(p.sources).to(DEV),
                    "out": torch.empty_like(sp)})
    eik.eik_solve_batched(dev)
    torch.cuda.synchronize()
    return [q["out"].cpu().numpy() for q in dev]


def _pinned_problems(probs, offset_out=False):
    host, keep = [], []
    pinned_speed = {}
    for i, p in enumerate(probs):
        key = id(p.speed)
        if key not in pinned_speed:
            pinned_speed[key] = torch.from_numpy(np.ascontiguousarray(p.speed)).pin_memory()
        n = p.speed.size
        if offset_out and i == 1:
            # an output that starts 8 bytes into its pinned allocation
            base = torch.full((n + 1,), -1.0, dtype=torch.float64).pin_memory()
            keep.append(base)
            out = base[1:].view(p.speed.shape)
        else:
            out = torch.full(p.speed.shape, -1.0, dtype=torch.float64).pin_memory()
        host.append({"speed": pinned_speed[key], "h": p.h, "sources": torch.from_numpy(p.sources),
                     "out": out})
    return host, keep


def test_pinned_batch_in_place_matches_device_and_oracle():
    probs = _batch_2d()
    want = _device_reference(probs)
    host, keep = _pinned_problems(probs, offset_out=True)
    assert all(q["out"].is_pinned() for q in host)
    eik.eik_solve_batched(host)
    for i, (q, w, p) in enumerate(zip(host, want, probs)):
        assert np.array_equal(_bits(q["out"].numpy()), _bits(w)), f"problem {i}"
        ref = oracle.fmm(p.speed, p.h, p.sources).t
        assert np.array_equal(_bits(q["out"].numpy()), _bits(ref)), f"problem {i} vs oracle"


def test_pageable_batch_matches_device():
    probs = _batch_2d()
    want = _device_reference(probs)
    host = [{"speed": np.ascontiguousarray(p.speed), "h": p.h, "sources": p.sources,
             "out": np.full(p.speed.shape, -1.0)} for p in probs]
    eik.eik_solve_batched(host)
    for i, (q, w) in enumerate(zip(host, want)):
        assert np.array_equal(_bits(q["out"]), _bits(w)), f"problem {i}"


def test_plan_over_pinned_buffers():
    probs = _batch_2d()
    want = _device_reference(probs)
    host, keep = _pinned_problems(probs, offset_out=True)
    plan = eik.Plan(host)
    for _ in range(2):
        for q in host:
            q["out"].fill_(-1.0)
        plan.enqueue()
        plan.status()
        for i, (q, w) in enumerate(zip(plan.problems, want)):
            assert np.array_equal(_bits(q["out"].numpy()), _bits(w)), f"problem {i}"
    plan.close()


def test_single_3d_grid_on_pinned_buffers():
    p = synth.random_problem(77, (19, 23, 21), n_src=2, contrast=5.0)
    speed = torch.from_numpy(np.ascontiguousarray(p.speed)).pin_memory()
    out = torch.full(p.speed.shape, -1.0, dtype=torch.float64).pin_memory()
    eik.solve(speed, p.h, p.sources, out=out)
    ref = oracle.fmm(p.speed, p.h, p.sources).t
    assert np.array_equal(_bits(out.numpy()), _bits(ref))

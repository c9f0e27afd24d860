"""GB300 (sm_103a) exactly monotone Eikonal solver: Python binding of include/eik.h.

The binding only marshals arguments to the C ABI of ``_libeik.so`` (built in
tree by ``build.py``); every step of the solve runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  If the library is
missing, importing the binding's functions raises instead of falling back to
anything else.

Names follow the C ABI: ``eik_solve``, ``eik_solve_batched``,
``eik_status_str``, ``eik_release``; ``solve`` and ``solve_batched`` are the
same calls taking tensors/arrays and returning the arrival times.

Method: arXiv 2103.05694 (Henriksen, You, Pingali), Algorithm 6 with the
exactly monotone rounding d-bar; result identical to Algorithm 2 (FMM) with
the same rounding (Theorem 1).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_libeik.so")

EIK_OK, EIK_EINVAL, EIK_ENOMEM, EIK_ECAPACITY, EIK_ETIMEOUT, EIK_ECUDA = range(6)


class EikOpts(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("k_delta", ctypes.c_double),
                ("capacity", ctypes.c_int64), ("timeout_ms", ctypes.c_int64),
                ("ctas_per_sm", ctypes.c_int), ("counters", ctypes.c_int),
                ("test_stall", ctypes.c_int), ("window", ctypes.c_int),
                ("band", ctypes.c_double), ("arith", ctypes.c_int), ("sched_flags", ctypes.c_int),
                ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_int64),
                ("tile", ctypes.c_int), ("update", ctypes.c_int),
                ("schedule", ctypes.c_int), ("reserved", ctypes.c_int)]

# opts["tile"] = k (1..5) selects TILE_SHAPES[ndim][k - 1]; 0 is automatic (16x16 for
# one 2D front, 16x8 for 2D batches of 8 or more sources, 4x4x4 in 3D)
TILE_SHAPES = {2: [(16, 16), (32, 8), (32, 4), (16, 8), (16, 4)],
               3: [(8, 8, 4), (16, 4, 4), (32, 4, 2), (8, 4, 4), (4, 4, 4)]}


TUNED_FIELDS = ("delta", "k_delta", "capacity", "ctas_per_sm", "window", "band", "arith", "tile")


def opts_dict(o: EikOpts) -> dict:
    """The scheduling fields of an EikOpts as a dict (for eik_* calls)."""
    return {k: getattr(o, k) for k in TUNED_FIELDS}


class EikTuneTrial(ctypes.Structure):
    _fields_ = [("opts", EikOpts), ("ms", ctypes.c_double), ("status", ctypes.c_int),
                ("reserved", ctypes.c_int)]


class EikStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("evals", "decreases", "good", "visits", "pushes", "stale_pops", "rounds",
                 "retries", "max_queue", "visit_ns", "idle_ns", "ctas", "trace_n")] + \
        [("detail", ctypes.c_int64 * 9), ("solve_ms", ctypes.c_double)]

    DETAIL = ["cyc_load", "cyc_a", "cyc_b", "cyc_c", "cyc_commit", "newton", "walk", "bisect",
              "dbar_calls"]

    def as_dict(self) -> dict:
        d = {n: getattr(self, n) for n, _ in self._fields_ if n != "detail"}
        d.update({k: int(self.detail[i]) for i, k in enumerate(self.DETAIL)})
        d["empty"] = d["evals"] - d["decreases"]
        d["bad"] = d["decreases"] - d["good"]
        return d


class EikProblem(ctypes.Structure):
    _fields_ = [("speed", ctypes.c_void_p), ("h", ctypes.c_double), ("ndim", ctypes.c_int),
                ("dims", ctypes.c_int64 * 3), ("src_idx", ctypes.c_void_p),
                ("src_t", ctypes.c_void_p), ("nsrc", ctypes.c_int64),
                ("out_t", ctypes.c_void_p)]


class EikError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{eik_status_str(status)}: {message}")
        self.status = status


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load _libeik.so (the CUDA path).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "`python -m paper_2103_05694_gb300.build` (needs nvcc)")
    L = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.eik_solve.argtypes = [vp, ctypes.c_double, ctypes.c_int, vp, vp, vp, i64, vp,
                            ctypes.POINTER(EikOpts), ctypes.POINTER(EikStats), vp]
    L.eik_solve.restype = ctypes.c_int
    L.eik_solve_batched.argtypes = [ctypes.POINTER(EikProblem), ctypes.c_int,
                                    ctypes.POINTER(EikOpts), ctypes.POINTER(EikStats), vp]
    L.eik_solve_batched.restype = ctypes.c_int
    L.eik_release.argtypes = []
    L.eik_release.restype = None
    L.eik_status_str.argtypes = [ctypes.c_int]
    L.eik_status_str.restype = ctypes.c_char_p
    L.eik_last_error.argtypes = []
    L.eik_last_error.restype = ctypes.c_char_p
    L.eik_abi_version.argtypes = []
    L.eik_abi_version.restype = ctypes.c_int
    L.eik_selftest.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64), vp]
    L.eik_selftest.restype = ctypes.c_int
    L.eik_solve_noalloc.argtypes = L.eik_solve.argtypes
    L.eik_solve_noalloc.restype = ctypes.c_int
    L.eik_plan_create.argtypes = [ctypes.POINTER(EikProblem), ctypes.c_int,
                                  ctypes.POINTER(EikOpts), ctypes.POINTER(vp)]
    L.eik_plan_create.restype = ctypes.c_int
    L.eik_plan_enqueue.argtypes = [vp, vp]
    L.eik_plan_enqueue.restype = ctypes.c_int
    L.eik_plan_status.argtypes = [vp, ctypes.POINTER(EikStats), vp]
    L.eik_plan_status.restype = ctypes.c_int
    L.eik_plan_destroy.argtypes = [vp]
    L.eik_plan_destroy.restype = None
    L.eik_adjoint.argtypes = [ctypes.POINTER(EikProblem), ctypes.c_int, ctypes.POINTER(vp),
                              ctypes.POINTER(vp), ctypes.POINTER(EikOpts),
                              ctypes.POINTER(EikStats), vp]
    L.eik_adjoint.restype = ctypes.c_int
    L.eik_kernel_launches.argtypes = []
    L.eik_kernel_launches.restype = ctypes.c_uint64
    L.eik_autotune.argtypes = [ctypes.POINTER(EikProblem), ctypes.c_int, ctypes.POINTER(EikOpts),
                               ctypes.c_int, ctypes.POINTER(EikOpts),
                               ctypes.POINTER(EikTuneTrial), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int), vp]
    L.eik_autotune.restype = ctypes.c_int
    L.eik_eval_update.argtypes = [ctypes.c_int, vp, ctypes.c_double, vp, vp, i64, vp, vp]
    L.eik_eval_update.restype = ctypes.c_int
    L.eik_residual.argtypes = [ctypes.POINTER(EikProblem), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double), vp]
    L.eik_residual.restype = ctypes.c_int
    L.eik_fp64_rate.argtypes = [i64, ctypes.POINTER(ctypes.c_double), vp]
    L.eik_fp64_rate.restype = ctypes.c_int
    L.eik_solve_slabs.argtypes = [vp, ctypes.c_double, ctypes.c_int, vp, vp, vp, i64, vp,
                                  ctypes.c_int, ctypes.POINTER(EikOpts), ctypes.POINTER(EikStats),
                                  ctypes.POINTER(ctypes.c_int), vp]
    L.eik_solve_slabs.restype = ctypes.c_int
    L.eik_sum_ordered.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, i64, vp]
    L.eik_sum_ordered.restype = ctypes.c_int
    _lib = L
    return L


EXPORTED = ["eik_solve", "eik_solve_batched", "eik_release", "eik_status_str", "eik_last_error",
            "eik_abi_version", "eik_selftest", "eik_solve_noalloc", "eik_plan_create",
            "eik_plan_enqueue", "eik_plan_status", "eik_plan_destroy", "eik_adjoint",
            "eik_kernel_launches", "eik_autotune", "eik_eval_update", "eik_residual",
            "eik_sum_ordered", "eik_solve_slabs", "eik_fp64_rate"]

SELFTEST_CHECKS = ["sub", "sq", "add", "G2", "G3", "dbar2", "dbar3", "group2x8", "group3x8",
                   "group2x4", "dbar2_fp64", "dbar3_fp64"]


def eik_selftest(n: int = 1 << 20, seed: int = 1, stream=None) -> dict:
    """Bit-exact check of the integer-pipe arithmetic against the FP64 unit, and
    of both d-bar paths against a bisection over the hardware G."""
    L = load_library()
    out = (ctypes.c_int64 * 32)()
    rc = L.eik_selftest(int(n), int(seed) & ((1 << 64) - 1), out, _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, "selftest failed to run")
    res = {k: int(out[i]) for i, k in enumerate(SELFTEST_CHECKS)}
    res["trials"] = int(out[15])
    res["first"] = {k: int(out[16 + i]) for i, k in enumerate(SELFTEST_CHECKS)}
    return res


def eik_status_str(status: int) -> str:
    return load_library().eik_status_str(int(status)).decode()


def eik_last_error() -> str:
    return load_library().eik_last_error().decode()


def eik_release() -> None:
    load_library().eik_release()


def eik_abi_version() -> int:
    return int(load_library().eik_abi_version())


def eik_kernel_launches() -> int:
    """Kernels the library has launched (or enqueued into a capture) so far."""
    return int(load_library().eik_kernel_launches())


def _make_opts(opts: dict | None) -> EikOpts | None:
    if not opts:
        return None
    names = {n for n, _ in EikOpts._fields_}
    unknown = sorted(set(opts) - names)
    if unknown:
        raise KeyError(f"unknown eik_opts fields {unknown}; known: {sorted(names)}")
    o = EikOpts()
    for k, v in opts.items():
        setattr(o, k, v)
    return o


def _stream_handle(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def eik_solve(speed_ptr: int, h: float, ndim: int, dims, src_ptr: int | None,
              src_t_ptr: int | None, nsrc: int, out_ptr: int, opts: dict | None = None,
              stream: int | None = None) -> dict:
    """Raw call: pointers are integers (device or host addresses)."""
    L = load_library()
    d = (ctypes.c_int64 * ndim)(*[int(x) for x in dims])
    st = EikStats()
    o = _make_opts(opts)
    rc = L.eik_solve(speed_ptr, float(h), int(ndim), d, src_ptr, src_t_ptr, int(nsrc), out_ptr,
                     ctypes.byref(o) if o is not None else None, ctypes.byref(st), stream)
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return st.as_dict()


def eik_solve_noalloc(speed_ptr: int, h: float, ndim: int, dims, src_ptr: int | None,
                      src_t_ptr: int | None, nsrc: int, out_ptr: int, opts: dict | None = None,
                      stream: int | None = None) -> dict:
    """Raw call of the allocation-free solve (device pointers only; at most
    2^20 cells, 2^15 tiles, 2048 sources).  For callers that may not allocate
    device memory."""
    L = load_library()
    d = (ctypes.c_int64 * ndim)(*[int(x) for x in dims])
    st = EikStats()
    o = _make_opts(opts)
    rc = L.eik_solve_noalloc(speed_ptr, float(h), int(ndim), d, src_ptr, src_t_ptr, int(nsrc),
                             out_ptr, ctypes.byref(o) if o is not None else None, ctypes.byref(st),
                             stream)
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return st.as_dict()


def _ptr(x):
    """Address of a contiguous torch tensor or numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


@dataclass
class SolveResult:
    t: object          # torch tensor or numpy array, same kind and device as `out`/speed
    stats: dict


def solve(speed, h: float, sources, src_t=None, out=None, opts: dict | None = None,
          stream=None) -> SolveResult:
    """Arrival times on a 2D/3D grid.  ``speed`` is a float64 torch tensor (any
    device) or numpy array, C-contiguous; ``sources`` flat int64 indices (same
    kind); ``out`` optional preallocated float64 output."""
    is_np = isinstance(speed, np.ndarray)
    if is_np:
        speed = np.ascontiguousarray(speed, dtype=np.float64)
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).reshape(-1))
        st = None if src_t is None else np.ascontiguousarray(np.asarray(src_t, np.float64).reshape(-1))
        if out is None:
            out = np.empty(speed.shape, dtype=np.float64)
    else:
        import torch
        if speed.dtype != torch.float64 or not speed.is_contiguous():
            raise ValueError("speed must be a contiguous float64 tensor")
        src = sources if isinstance(sources, torch.Tensor) else torch.as_tensor(
            np.asarray(sources, dtype=np.int64))
        src = src.to(device=speed.device, dtype=torch.int64).contiguous().reshape(-1)
        st = None
        if src_t is not None:
            st = src_t if isinstance(src_t, torch.Tensor) else torch.as_tensor(
                np.asarray(src_t, dtype=np.float64))
            st = st.to(device=speed.device, dtype=torch.float64).contiguous().reshape(-1)
        if out is None:
            out = torch.empty_like(speed)
    stats = eik_solve(_ptr(speed), h, speed.ndim, speed.shape, _ptr(src), _ptr(st),
                      int(src.shape[0]), _ptr(out), opts, _stream_handle(stream) if not is_np
                      else None)
    return SolveResult(out, stats)


def eik_solve_batched(problems: list[dict], opts: dict | None = None, stream=None) -> dict:
    """Batched call.  Each problem dict holds speed, sources, optional src_t, out
    (torch tensors on the device or in host memory, or numpy arrays; host
    buffers are staged inside the call) and h.  All problems run in one
    persistent launch."""
    L = load_library()
    arr = _problem_array(problems)
    st = EikStats()
    o = _make_opts(opts)
    rc = L.eik_solve_batched(arr, len(problems), ctypes.byref(o) if o is not None else None,
                             ctypes.byref(st), _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return st.as_dict()


def solve_batched(problems: list[dict], opts: dict | None = None, stream=None) -> dict:
    """Like eik_solve_batched, allocating ``out`` where missing."""
    import torch
    for p in problems:
        if p.get("out") is None:
            p["out"] = torch.empty_like(p["speed"])
        src = p["sources"]
        if not isinstance(src, torch.Tensor):
            src = torch.as_tensor(np.asarray(src, dtype=np.int64))
        p["sources"] = src.to(device=p["speed"].device, dtype=torch.int64).contiguous()
        if p.get("src_t") is not None and not isinstance(p["src_t"], torch.Tensor):
            p["src_t"] = torch.as_tensor(np.asarray(p["src_t"], np.float64)).to(p["speed"].device)
    return eik_solve_batched(problems, opts, stream)


def _problem_array(problems: list[dict]):
    arr = (EikProblem * len(problems))()
    for i, p in enumerate(problems):
        sp = p["speed"]
        arr[i].speed = _ptr(sp)
        arr[i].h = float(p["h"])
        arr[i].ndim = sp.ndim
        for k in range(3):
            arr[i].dims[k] = int(sp.shape[k]) if k < sp.ndim else 1
        arr[i].src_idx = _ptr(p["sources"])
        arr[i].src_t = _ptr(p.get("src_t"))
        src = p["sources"]
        arr[i].nsrc = int(src.numel() if hasattr(src, "numel") else np.asarray(src).size)
        arr[i].out_t = _ptr(p["out"])
    return arr


def eik_plan_create(problems: list[dict], opts: dict | None = None) -> int:
    """Prepare a batch (torch CUDA tensors: speed, sources, optional src_t, out;
    and h).  Returns the plan handle."""
    L = load_library()
    arr = _problem_array(problems)
    o = _make_opts(opts)
    h = ctypes.c_void_p()
    rc = L.eik_plan_create(arr, len(problems), ctypes.byref(o) if o is not None else None,
                           ctypes.byref(h))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return h.value


def eik_plan_enqueue(plan: int, stream=None) -> None:
    rc = load_library().eik_plan_enqueue(plan, _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())


def eik_plan_status(plan: int, stream=None) -> dict:
    st = EikStats()
    rc = load_library().eik_plan_status(plan, ctypes.byref(st), _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return st.as_dict()


def eik_plan_destroy(plan: int) -> None:
    load_library().eik_plan_destroy(plan)


class Plan:
    """A batch of problems solved together in one persistent launch per solve.
    ``enqueue`` only enqueues device work (no allocation, no host wait), so it
    can be captured in a torch.cuda.CUDAGraph and replayed."""

    def __init__(self, problems: list[dict], opts: dict | None = None):
        import torch
        for p in problems:
            if p.get("out") is None:
                p["out"] = torch.empty_like(p["speed"])
            src = p["sources"]
            if not isinstance(src, torch.Tensor):
                src = torch.as_tensor(np.asarray(src, dtype=np.int64))
            p["sources"] = src.to(device=p["speed"].device, dtype=torch.int64).contiguous()
        self.problems = problems          # keeps the tensors alive
        self.handle = eik_plan_create(problems, opts)

    def enqueue(self, stream=None) -> None:
        eik_plan_enqueue(self.handle, stream)

    def status(self, stream=None) -> dict:
        return eik_plan_status(self.handle, stream)

    def close(self) -> None:
        if self.handle:
            eik_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# eik_adjoint schedule (opts["sched_flags"] bits 3-4): cells level by level
# between grid barriers, or tiles in shared memory handed over through a queue
ADJ_LEVELS = 1 << 3
ADJ_TILES = 2 << 3
# opts["sched_flags"] bit 6: the "speed" arrays hold slowness s (v = fl(1/s) on the
# device); bit 7 (eik_adjoint): problems sharing a gradient array receive the sum of
# their gradients in problem order
SLOWNESS_INPUT = 1 << 6
SUM_SHARED_GRADIENTS = 1 << 7


def eik_adjoint(problems: list[dict], dL_dt: list, dL_ds: list, opts: dict | None = None,
                stream=None) -> dict:
    """d(loss)/d(slowness) through the solved fields ``problems[i]["out"]``.
    dL_dt[i] (tensor or None) is d(loss)/d(t); dL_ds[i] (tensor) receives the
    gradient.  All torch CUDA tensors."""
    L = load_library()
    arr = _problem_array(problems)
    n = len(problems)
    gt = (ctypes.c_void_p * n)(*[_ptr(x) for x in dL_dt])
    gs = (ctypes.c_void_p * n)(*[_ptr(x) for x in dL_ds])
    st = EikStats()
    o = _make_opts(opts)
    rc = L.eik_adjoint(arr, n, gt, gs, ctypes.byref(o) if o is not None else None,
                       ctypes.byref(st), _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return st.as_dict()


def eik_autotune(problems: list[dict], base: dict | None = None, repeats: int = 2,
                 max_trials: int = 128, stream=None) -> tuple[dict, list[dict]]:
    """Pick tile shape, bucket width, look-ahead, band, CTAs per SM and frontier
    capacity for this batch by timing it (torch CUDA tensors as in
    eik_solve_batched).  Returns (options, trials); every trial reproduced the
    same bits."""
    L = load_library()
    arr = _problem_array(problems)
    best = EikOpts()
    tr = (EikTuneTrial * max_trials)()
    nt = ctypes.c_int(0)
    o = _make_opts(base)
    rc = L.eik_autotune(arr, len(problems), ctypes.byref(o) if o is not None else None,
                        int(repeats), ctypes.byref(best), tr, max_trials, ctypes.byref(nt),
                        _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    trials = [dict(opts_dict(tr[i].opts), ms=tr[i].ms, status=tr[i].status)
              for i in range(nt.value)]
    return opts_dict(best), trials


UPDATE_FORMS = {"dbar": 0, "dtilde": 1, "dhat": 2, "newton": 3}
# opts["sched_flags"] bit 5: with an explicit form, a recomputed value that differs
# (up or down) replaces the cell's and re-activates its neighbours
TRACK_CHANGES = 1 << 5


def eik_eval_update(form: int, speed, h: float, t_h, t_v, out=None, stream=None):
    """One application of the update per point (form 0 = d-bar, 1 = d-tilde,
    2 = d-hat; 2D).  torch CUDA float64 tensors of one shape; returns ``out``."""
    import torch
    if out is None:
        out = torch.empty_like(speed)
    L = load_library()
    rc = L.eik_eval_update(int(form), _ptr(speed), float(h), _ptr(t_h), _ptr(t_v),
                           int(speed.numel()), _ptr(out), _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return out


def eik_residual(problem: dict, form: int = 0, stream=None) -> tuple[int, float]:
    """Table 3 residual of problem["out"] (device tensors as in eik_solve_batched):
    (cells not fixed under the update, largest relative change)."""
    L = load_library()
    arr = _problem_array([problem])
    bad = ctypes.c_int64(0)
    rel = ctypes.c_double(0.0)
    rc = L.eik_residual(arr, int(form), ctypes.byref(bad), ctypes.byref(rel),
                        _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return int(bad.value), float(rel.value)


def solve_slabs(speed, h: float, sources, nslabs: int, src_t=None, out=None,
                opts: dict | None = None, stream=None) -> SolveResult:
    """The grid split into ``nslabs`` slabs along its outermost axis, solved by
    epochs with halo exchange (eik_solve_slabs; same bits as ``solve``).  torch
    CUDA float64 tensors; stats["epochs"] is the number of epochs."""
    import torch
    if speed.dtype != torch.float64 or not speed.is_contiguous() or not speed.is_cuda:
        raise ValueError("speed must be a contiguous float64 CUDA tensor")
    src = sources if isinstance(sources, torch.Tensor) else torch.as_tensor(
        np.asarray(sources, dtype=np.int64))
    src = src.to(device=speed.device, dtype=torch.int64).contiguous().reshape(-1)
    st_t = None
    if src_t is not None:
        st_t = torch.as_tensor(src_t, dtype=torch.float64).to(speed.device).contiguous().reshape(-1)
    if out is None:
        out = torch.empty_like(speed)
    stats = eik_solve_slabs(_ptr(speed), h, speed.ndim, speed.shape, _ptr(src), _ptr(st_t),
                            int(src.numel()), _ptr(out), nslabs, opts, _stream_handle(stream))
    return SolveResult(out, stats)


def eik_solve_slabs(speed_ptr: int, h: float, ndim: int, dims, src_ptr: int | None,
                    src_t_ptr: int | None, nsrc: int, out_ptr: int, nslabs: int,
                    opts: dict | None = None, stream: int | None = None) -> dict:
    """Raw call of the slab-decomposed solve (device speed and out); the stats
    dict adds "epochs"."""
    L = load_library()
    d = (ctypes.c_int64 * ndim)(*[int(x) for x in dims])
    st = EikStats()
    ep = ctypes.c_int(0)
    o = _make_opts(opts)
    rc = L.eik_solve_slabs(speed_ptr, float(h), int(ndim), d, src_ptr, src_t_ptr, int(nsrc),
                           out_ptr, int(nslabs), ctypes.byref(o) if o is not None else None,
                           ctypes.byref(st), ctypes.byref(ep), stream)
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    stats = st.as_dict()
    stats["epochs"] = int(ep.value)
    return stats


def eik_fp64_rate(iters: int = 1 << 16, stream=None) -> float:
    """Measured FP64 add throughput of the current device (thread instructions/s)."""
    r = ctypes.c_double(0.0)
    rc = load_library().eik_fp64_rate(int(iters), ctypes.byref(r), _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, "eik_fp64_rate")
    return float(r.value)


def eik_sum_ordered(srcs: list, out, stream=None):
    """out = +0 + srcs[0] + srcs[1] + ... in list order, each addition rounded to
    nearest (torch CUDA float64 tensors of out's size; the library's kernel)."""
    n = len(srcs)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[_ptr(x) for x in srcs])
    rc = load_library().eik_sum_ordered(ptrs, n, _ptr(out), int(out.numel()),
                                        _stream_handle(stream))
    if rc != EIK_OK:
        raise EikError(rc, eik_last_error())
    return out


def _make_eikonal_fn():
    import torch

    class EikonalFn(torch.autograd.Function):
        """Arrival times of several source sets on one slowness field, and the
        exact adjoint as backward.

        forward(slowness, h, sources): slowness (float64 CUDA tensor, 2D or 3D),
        sources a list of int64 tensors (flat indices), one solve per entry, all
        in one persistent launch; the library converts slowness to speed
        (v = fl(1/s)) on the device.  Returns t with shape (len(sources), *grid).
        backward: d(loss)/d(slowness) summed over the solves in source order by
        the library (eik_adjoint with SUM_SHARED_GRADIENTS).  The binding only
        allocates and passes pointers."""

        @staticmethod
        def forward(ctx, slowness, h, sources):
            if slowness.dtype != torch.float64 or not slowness.is_contiguous():
                raise ValueError("slowness must be a contiguous float64 tensor")
            t = torch.empty((len(sources),) + tuple(slowness.shape), dtype=slowness.dtype,
                            device=slowness.device)
            probs = [{"speed": slowness, "h": h, "sources": src, "out": t[i]}
                     for i, src in enumerate(sources)]
            eik_solve_batched(probs, {"sched_flags": SLOWNESS_INPUT})
            ctx.save_for_backward(slowness, t)
            ctx.h = h
            ctx.sources = sources
            return t

        @staticmethod
        def backward(ctx, grad_t):
            slowness, t = ctx.saved_tensors
            grad_t = grad_t.contiguous()
            grad = torch.empty_like(slowness)
            probs = [{"speed": slowness, "h": ctx.h, "sources": src, "out": t[i]}
                     for i, src in enumerate(ctx.sources)]
            eik_adjoint(probs, [grad_t[i] for i in range(len(probs))], [grad] * len(probs),
                        {"sched_flags": SLOWNESS_INPUT | SUM_SHARED_GRADIENTS})
            return grad, None, None

    return EikonalFn


_eikonal_fn = None


def eikonal(slowness, h: float, sources):
    """Differentiable batched solve (see EikonalFn)."""
    global _eikonal_fn
    if _eikonal_fn is None:
        _eikonal_fn = _make_eikonal_fn()
    return _eikonal_fn.apply(slowness, h, list(sources))

"""CPU oracle for the exactly monotone first-order Eikonal update (arXiv 2103.05694).

TEST INFRASTRUCTURE ONLY.  The plain, slow, single-threaded C definition in
``oracle.c`` (FP64, no FMA contraction) that the CUDA path is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Functions and the passages they follow:

* ``dtilde`` -- the classical explicit root d-tilde (Loss of Monotonicity section, Table 1).
* ``dhat`` -- the rearranged explicit root d-hat (Mitigation Strategies, Table 2).
* ``cell_c`` -- c = fl(fl(h/v)^2), the right-hand side of Eq. difference_as_root.
* ``G``, ``dbar``, ``dbar_bisect`` -- the exactly monotone rounding d-bar
  (Achieving Exact Monotonicity section), two independent searches.
* ``fmm`` -- the fast marching method, Algorithm 2, binary heap.
* ``sweep`` -- topology-driven solver, Algorithm 4 (mode 0) and the fast sweeping
  method, Algorithm 5 (mode 1).
* ``relax_order`` -- relaxation in a caller-given order (Theorem 1).
* ``residual`` -- the fixed-point residual of Table 3 (d-bar, or in 2D Algorithm 1
  with the explicit roots d-tilde / d-hat / d-hat then Newton: ``form`` 1 / 2 / 3).
* ``update_form`` -- one application of Algorithm 1 with d-tilde (form 1), d-hat
  (form 2), d-hat followed by Newton's method on alpha = 0 (form 3) or d-bar
  (form 0) (Mitigation Strategies and Achieving Exact Monotonicity sections).
* ``adjoint`` -- d(loss)/d(slowness) through the fixed point (not in the paper:
  implicit differentiation of the real-arithmetic local equations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liborc.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile oracle.c into _liborc.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrcStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("pops", "stale", "evals", "decreases", "increases", "order_breaks", "sweeps")]

    def as_dict(self) -> dict:
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None
_d = ctypes.c_double
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_dtilde.argtypes = [_d, _d, _d, _d]; L.orc_dtilde.restype = _d
        L.orc_dhat.argtypes = [_d, _d, _d, _d]; L.orc_dhat.restype = _d
        L.orc_cell_c.argtypes = [_d, _d]; L.orc_cell_c.restype = _d
        L.orc_G.argtypes = [_d, _p, ctypes.c_int]; L.orc_G.restype = _d
        L.orc_dbar.argtypes = [_p, ctypes.c_int, _d, _d]; L.orc_dbar.restype = _d
        L.orc_dbar_bisect.argtypes = [_p, ctypes.c_int, _d]; L.orc_dbar_bisect.restype = _d
        L.orc_fmm.argtypes = [ctypes.c_int, _p, _p, _d, _p, _p, _i64, _p, ctypes.POINTER(OrcStats)]
        L.orc_fmm.restype = ctypes.c_int
        L.orc_sweep.argtypes = [ctypes.c_int, _p, _p, _d, _p, _p, _i64, ctypes.c_int, _p,
                                ctypes.POINTER(OrcStats)]
        L.orc_sweep.restype = ctypes.c_int
        L.orc_relax_order.argtypes = [ctypes.c_int, _p, _p, _d, _p, _p, _i64, _p, _i64, _p,
                                      ctypes.POINTER(OrcStats)]
        L.orc_relax_order.restype = ctypes.c_int
        L.orc_residual.argtypes = [ctypes.c_int, _p, _p, _d, _p, _p, _i64, _p,
                                   ctypes.POINTER(_d)]
        L.orc_residual.restype = _i64
        L.orc_residual_form.argtypes = [ctypes.c_int, ctypes.c_int, _p, _p, _d, _p, _p, _i64, _p,
                                        ctypes.POINTER(_d)]
        L.orc_residual_form.restype = _i64
        L.orc_update_form.argtypes = [ctypes.c_int, _d, _d, _d, _d]
        L.orc_update_form.restype = _d
        L.orc_adjoint.argtypes = [ctypes.c_int, _p, _p, _d, _p, _i64, _p, _p, _p, _p]
        L.orc_adjoint.restype = ctypes.c_int
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_p)


def dtilde(v: float, h: float, tH: float, tV: float) -> float:
    return lib().orc_dtilde(v, h, tH, tV)


def dhat(v: float, h: float, tH: float, tV: float) -> float:
    return lib().orc_dhat(v, h, tH, tV)


def cell_c(v: float, h: float) -> float:
    return lib().orc_cell_c(v, h)


def G(tau: float, a) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_G(tau, _ptr(a), a.size)


def dbar(a, r: float, c: float) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_dbar(_ptr(a), a.size, r, c)


def dbar_bisect(a, c: float) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().orc_dbar_bisect(_ptr(a), a.size, c)


def _grid_args(speed: np.ndarray, sources, src_t):
    speed = np.ascontiguousarray(speed, dtype=np.float64)
    dims = np.asarray(speed.shape, dtype=np.int64)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int64).reshape(-1))
    st = None if src_t is None else np.ascontiguousarray(np.asarray(src_t, dtype=np.float64).reshape(-1))
    return speed, dims, src, st


@dataclass
class OracleResult:
    t: np.ndarray
    stats: dict


def fmm(speed: np.ndarray, h: float, sources, src_t=None) -> OracleResult:
    """Arrival times by the fast marching method (Algorithm 2).  ``sources`` are
    flat C-order cell indices; ``src_t`` their times (default 0)."""
    speed, dims, src, st = _grid_args(speed, sources, src_t)
    t = np.empty(speed.shape, dtype=np.float64)
    s = OrcStats()
    rc = lib().orc_fmm(speed.ndim, _ptr(dims), _ptr(speed), h, _ptr(src), _ptr(st), src.size,
                       _ptr(t), ctypes.byref(s))
    if rc != 0:
        raise RuntimeError("orc_fmm failed")
    return OracleResult(t, s.as_dict())


def sweep(speed: np.ndarray, h: float, sources, src_t=None, mode: int = 0) -> OracleResult:
    """Topology-driven solver: mode 0 = Algorithm 4, mode 1 = Algorithm 5 (FSM)."""
    speed, dims, src, st = _grid_args(speed, sources, src_t)
    t = np.empty(speed.shape, dtype=np.float64)
    s = OrcStats()
    rc = lib().orc_sweep(speed.ndim, _ptr(dims), _ptr(speed), h, _ptr(src), _ptr(st), src.size,
                         mode, _ptr(t), ctypes.byref(s))
    if rc != 0:
        raise RuntimeError("orc_sweep failed")
    return OracleResult(t, s.as_dict())


def relax_order(speed: np.ndarray, h: float, sources, perm, src_t=None) -> OracleResult:
    """Repeated passes over the cells in the order ``perm`` until nothing changes."""
    speed, dims, src, st = _grid_args(speed, sources, src_t)
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int64).reshape(-1))
    t = np.empty(speed.shape, dtype=np.float64)
    s = OrcStats()
    rc = lib().orc_relax_order(speed.ndim, _ptr(dims), _ptr(speed), h, _ptr(src), _ptr(st),
                               src.size, _ptr(perm), perm.size, _ptr(t), ctypes.byref(s))
    if rc != 0:
        raise RuntimeError("orc_relax_order failed")
    return OracleResult(t, s.as_dict())


def update_form(form: int, v: float, h: float, tH: float, tV: float) -> float:
    """Algorithm 1 with root d-tilde (1), d-hat (2), d-hat then Newton (3) or d-bar (0)."""
    return lib().orc_update_form(int(form), v, h, tH, tV)


def residual(speed: np.ndarray, h: float, sources, t: np.ndarray, src_t=None, form: int = 0):
    """Table 3 residual of a field: (number of cells that are not fixed under the
    operator, largest relative difference).  ``form`` as in update_form (1-3:
    2D only)."""
    speed, dims, src, st = _grid_args(speed, sources, src_t)
    t = np.ascontiguousarray(t, dtype=np.float64)
    if t.shape != speed.shape:
        raise ValueError("shape mismatch")
    mr = _d(0.0)
    bad = lib().orc_residual_form(int(form), speed.ndim, _ptr(dims), _ptr(speed), h, _ptr(src),
                                  _ptr(st), src.size, _ptr(t), ctypes.byref(mr))
    if bad < 0:
        raise RuntimeError("orc_residual failed")
    return int(bad), float(mr.value)


def adjoint(speed: np.ndarray, h: float, sources, t: np.ndarray, dL_dt: np.ndarray):
    """(lambda, dL/ds) for the fixed point t of the problem and g = dL/dt."""
    speed, dims, src, _ = _grid_args(speed, sources, None)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.ascontiguousarray(dL_dt, dtype=np.float64)
    lam = np.empty(speed.shape)
    gs = np.empty(speed.shape)
    rc = lib().orc_adjoint(speed.ndim, _ptr(dims), _ptr(speed), h, _ptr(src), src.size, _ptr(t),
                           _ptr(g), _ptr(lam), _ptr(gs))
    if rc != 0:
        raise RuntimeError("orc_adjoint failed")
    return lam, gs

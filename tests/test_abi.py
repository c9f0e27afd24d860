"""The C-ABI library builds, loads and exports every symbol include/eik.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_2103_05694_gb300 as eik
from paper_2103_05694_gb300 import build as eikbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "eik.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eik_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    eikbuild.build()
    return ctypes.CDLL(eikbuild.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("eik_solve", "eik_solve_batched", "eik_status_str", "eik_release"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_the_abi():
    for name in declared_functions():
        assert name in eik.EXPORTED, name
        assert callable(getattr(eik, name)), name


def test_status_strings_without_gpu(lib):
    lib.eik_status_str.restype = ctypes.c_char_p
    lib.eik_status_str.argtypes = [ctypes.c_int]
    assert lib.eik_status_str(0) == b"EIK_OK"
    assert lib.eik_status_str(3) == b"EIK_ECAPACITY"
    lib.eik_abi_version.restype = ctypes.c_int
    assert lib.eik_abi_version() == 108


def test_struct_layouts_match_header():
    # eik_opts: double, double, int64, int64, 4 x int, double, 2 x int, ptr, int64, 4 x int
    assert ctypes.sizeof(eik.EikOpts) == 96
    assert ctypes.sizeof(eik.EikStats) == 23 * 8
    # eik_problem: ptr, double, int(+pad), int64[3], ptr, ptr, int64, ptr
    assert ctypes.sizeof(eik.EikProblem) == 8 + 8 + 8 + 24 + 8 + 8 + 8 + 8


def test_missing_library_fails_loudly(tmp_path):
    saved = eik._lib
    try:
        eik._lib = None
        with pytest.raises(RuntimeError):
            eik.load_library(str(tmp_path / "nope.so"))
    finally:
        eik._lib = saved


def test_kernel_launch_counter_without_gpu(lib):
    lib.eik_kernel_launches.restype = ctypes.c_uint64
    assert lib.eik_kernel_launches() == 0      # nothing launched in this process yet


def test_tune_trial_layout():
    # eik_tune_trial: eik_opts, double, int, int
    assert ctypes.sizeof(eik.EikTuneTrial) == 96 + 8 + 4 + 4


def test_unknown_option_names_are_rejected():
    with pytest.raises(KeyError):
        eik._make_opts({"bnd": 4.0})
    o = eik._make_opts({"band": 4.0, "tile": 1, "schedule": 2})
    assert o.band == 4.0 and o.tile == 1 and o.schedule == 2

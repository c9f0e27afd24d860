"""Host logic of bench.py that runs without a GPU: the clock-sample summary, the
roofline arithmetic, the options a command line turns into, and the all-cores
oracle baseline (spawned worker processes meeting at a barrier)."""
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    s = bench.ClockSampler(0)
    s.lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, N/A, 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = s.summary()
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    s.lines = ["0, 1500, 2070, 1400, 0x8, Not Active, Active, Not Active, Not Active"]
    assert bench.ClockSampler.summary(s)["reasons"] == ["hw_thermal_slowdown"]
    s.lines = []
    assert s.summary()["reasons"] == ["no samples"]


def test_roofline_uses_the_measured_copy_peak():
    peak, kind = bench.measured_peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    r = bench.roofline(1_000_000, 2.0, 123, "k")
    # 24 algorithmic bytes per useful update over the launch time
    assert r["bytes_per_launch"] == 24_000_000
    assert abs(r["achieved"] - 24e6 / 2e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-15
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 123


def test_command_line_options():
    ns = types.SimpleNamespace(k_delta=2.0, ctas_per_sm=0, window=8, band=0.0, tile=4,
                               update=2, track_changes=True, schedule=0)
    from paper_2103_05694_gb300 import TRACK_CHANGES
    assert bench.make_opts(ns) == {"k_delta": 2.0, "window": 8, "tile": 4, "update": 2,
                                   "sched_flags": TRACK_CHANGES}
    ns = types.SimpleNamespace(k_delta=0.0, ctas_per_sm=0, window=0, band=0.0, tile=0,
                               update=0, track_changes=False, schedule=0)
    assert bench.make_opts(ns) == {}


@pytest.mark.parametrize("argv", [["--problems", "89"], ["--problems", "-1"],
                                  ["--workload", "checker_3d", "--problems", "4"]])
def test_reduced_batch_option_is_checked(argv, monkeypatch):
    """--problems takes 1..88 and the batch only; it stops before any GPU work."""
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    with pytest.raises(SystemExit, match="--problems takes 1..88"):
        bench.main()


@pytest.mark.slow
def test_all_cores_oracle_baseline_runs_every_core():
    """One spawned process per host core solves its share of the tomography
    sources (FMM + adjoint); the job's time is the slowest process's."""
    args = types.SimpleNamespace(workload="tomography_2d")
    r = bench.cpu_baseline_all_cores(args, per_unit_s=10.0, seconds=0.5)
    cores = len(os.sched_getaffinity(0))
    assert r["cores"] == cores and r["kind"] == "oracle" and r["value"] > 0
    assert f"on {cores} host cores" in r["sample"]


def test_fp64_roofline_arithmetic():
    """FP64 instructions per launch = instructions per evaluation (ncu) x the live
    evaluation count; achieved over the kernel time, against the measured rate."""
    fake = types.SimpleNamespace(eik=types.SimpleNamespace(eik_fp64_rate=lambda: 5.0e11))
    saved = dict(bench.MEASURED_FP64_PER_EVAL)
    try:
        bench.MEASURED_FP64_PER_EVAL[3] = 20.0
        r = bench.roofline_fp64(fake, 1_000_000, 4.0, 3, "k")
        assert r["bound"] == "fp64" and r["peak"] == 500.0
        assert abs(r["achieved"] - 20.0 * 1e6 / 4e-3 / 1e9) < 1e-9
        assert abs(r["frac"] - r["achieved"] / 500.0) < 1e-15
        bench.MEASURED_FP64_PER_EVAL[3] = None
        r = bench.roofline_fp64(fake, 1_000_000, 4.0, 3, "k")
        assert r["achieved"] is None and r["frac"] is None and r["peak"] == 500.0
    finally:
        bench.MEASURED_FP64_PER_EVAL.clear()
        bench.MEASURED_FP64_PER_EVAL.update(saved)

"""Benchmark: useful grid-point updates per second of the exact Eikonal solve.

One step = one pass of the whole hot path on one grid: per-cell constants
r = fl(h/v) and t = +inf, source seeding, and the persistent bucket-scheduled
relaxation to the exact fixed point (Algorithm 6 with the exactly monotone
d-bar of arXiv 2103.05694).  Default workload: the 2D layered seismic-like
model, 2301 x 751 cells, h = 4 m, one surface source (synthetic; it stands in
for the paper's Marmousi section).

Prints one JSON line (rank 0).  Arms:
  default          the CUDA library through its C ABI, inputs resident in HBM;
  --impl reference the CPU oracle (single-threaded fast marching, Algorithm 2)
                   timed on the host cores on a bounded sample of the workload.
Multi-GPU (torchrun): every rank solves its own replica (the single-grid path
does not shard: replicas only, weak scaling); no collective touches the data.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "useful grid-point updates/s and % HBM roofline (bit-exact vs FP64 FMM oracle)"
UNIT = "updates/s"
B_ALG = 24          # algorithmic bytes per useful update: read r once, read t once, write t once
L2_FLUSH_BYTES = 512 << 20


def workloads():
    return {
        "1": ("2d_129x129_const (config 1)", synth.config1),
        "2": ("2d_2301x751_layered (config 2)", synth.config2),
        "3": ("3d_256cube_smooth_checker (config 3)", synth.config3),
    }


def scaled_layered(scale: float):
    """The layered 2D model at a fraction of its extent per axis (profiling cases)."""
    nx, nz = max(32, round(2301 * scale)), max(8, round(751 * scale))
    speed = synth.layered_section(nx, nz, 4.0, seed=2)
    src = np.array([nx // 2], dtype=np.int64)
    return synth.Problem(f"2d_{nx}x{nz}_layered", speed, 4.0, src, np.zeros(1), {})


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args, wl_name, prob, useful):
    """The CPU oracle, as it stands, on bounded samples of the same workload."""
    import oracle
    oracle.build()
    if args.rank != 0:
        return
    budget_s = args.ref_seconds
    per_step = []
    for _ in range(args.warmup):
        oracle.fmm(prob.speed, prob.h, prob.sources, prob.src_t)
    n_solves = 0
    t_all0 = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.fmm(prob.speed, prob.h, prob.sources, prob.src_t)
        per_step.append(time.perf_counter() - t0)
        n_solves += 1
        if time.perf_counter() - t_all0 > budget_s:
            break
    useful_ref = int(np.isfinite(r.t).sum()) - len(np.unique(prob.sources))
    total = sum(per_step)
    value = useful_ref * len(per_step) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": len(per_step), "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(per_step), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl_name, "cells": prob.ncells, "sources": int(len(prob.sources))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{len(per_step)} full single-threaded FMM solves of the "
                                   f"workload (stopping after {budget_s:.0f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(prob, seconds):
    import oracle
    oracle.build()
    times = []
    t_all = time.perf_counter()
    r = None
    while True:
        t0 = time.perf_counter()
        r = oracle.fmm(prob.speed, prob.h, prob.sources, prob.src_t)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > seconds:
            break
    useful = int(np.isfinite(r.t).sum()) - len(np.unique(prob.sources))
    return {"value": useful * len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} full single-threaded FMM solves of the workload "
                      f"({sum(times):.1f} s of CPU time)", "ms_per_solve": 1e3 * sum(times) / len(times)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="2", choices=sorted(workloads()))
    ap.add_argument("--scale", type=float, default=1.0,
                    help="config 2 only: fraction of the extent per axis (profiling)")
    ap.add_argument("--k-delta", type=float, default=0.0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="ncu dram bytes per launch of the solve kernel, if measured")
    args = ap.parse_args()
    args.rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus and world > 1:
        args.gpus = world

    wl_name, make = workloads()[args.config]
    if args.config == "2" and args.scale != 1.0:
        prob = scaled_layered(args.scale)
        wl_name = prob.name + " (config 2 scaled)"
    else:
        prob = make()
    useful = prob.ncells - len(np.unique(prob.sources))   # every cell is reachable

    if args.impl == "reference":
        run_reference(args, wl_name, prob, useful)
        return

    import torch
    import paper_2103_05694_gb300 as eik
    from paper_2103_05694_gb300 import build as eikbuild
    eikbuild.build()
    eik.load_library()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    opts = {}
    if args.k_delta > 0:
        opts["k_delta"] = args.k_delta
    if args.ctas_per_sm > 0:
        opts["ctas_per_sm"] = args.ctas_per_sm
    speed = torch.from_numpy(prob.speed).to(dev)
    src = torch.from_numpy(prob.sources).to(dev)
    out = torch.empty_like(speed)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    # correctness gate on the timed configuration: the exact fixed point
    st = eik.solve(speed, prob.h, src, out=out, opts=dict(opts, counters=1)).stats
    torch.cuda.synchronize(dev)
    assert st["good"] == useful, (st, useful)

    for _ in range(args.warmup):
        eik.solve(speed, prob.h, src, out=out, opts=opts)
        flush.zero_()
    torch.cuda.synchronize(dev)

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    solve_ms = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            evs[i][0].record(stream)
            s = eik.solve(speed, prob.h, src, out=out, opts=opts).stats
            evs[i][1].record(stream)
            solve_ms.append(s["solve_ms"])
            flush.zero_()            # L2 flush between timed steps (outside the events)
        torch.cuda.synchronize(dev)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    n = args.gpus
    value = useful * args.steps * n / (total_ms / 1e3)
    evals_per_step = st["evals"]

    # end to end through the C ABI with host buffers (copies inside the call)
    h_speed = torch.from_numpy(prob.speed).pin_memory()
    h_out = torch.empty(prob.speed.shape, dtype=torch.float64).pin_memory()
    h_src = prob.sources.copy()
    e2e_steps = max(3, min(args.steps, 30))
    for _ in range(2):
        eik.eik_solve(h_speed.data_ptr(), prob.h, prob.speed.ndim, prob.speed.shape,
                      h_src.ctypes.data, None, len(h_src), h_out.data_ptr(), opts or None,
                      stream.cuda_stream)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        eik.eik_solve(h_speed.data_ptr(), prob.h, prob.speed.ndim, prob.speed.shape,
                      h_src.ctypes.data, None, len(h_src), h_out.data_ptr(), opts or None,
                      stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    assert np.array_equal(h_out.numpy(), out.cpu().numpy())
    e2e_value = useful * n / (e2e_ms / 1e3)

    peak, peak_kind = measured_peaks()
    kern_ms = statistics.mean(solve_ms)
    achieved = B_ALG * useful / (kern_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": args.traffic_bytes,
            "kernel": "persistent_kernel (tile relaxation + bucket scheduler)",
            "kernel_ms": kern_ms, "bytes_per_launch": B_ALG * useful,
            "peak_kind": f"{peak_kind} copy bandwidth"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": n, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl_name, "cells": prob.ncells, "h": prob.h,
                   "sources": int(len(prob.sources)), "parallelism": f"replicas x{n}",
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)",
                   "opts": opts},
        "grid_point_updates_per_s": evals_per_step * args.steps * n / (total_ms / 1e3),
        "work_per_step": {k: st[k] for k in ("evals", "decreases", "good", "empty", "bad",
                                             "visits", "pushes", "stale_pops", "rounds")},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(prob.speed.nbytes + h_src.nbytes),
                "d2h_bytes_per_step": int(prob.speed.nbytes)},
        "gpu_launches": 4 * args.steps,
        "clocks": clk.summary(),
    }
    if args.rank == 0 and n == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, args.cpu_seconds)
    if args.rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

"""Benchmark: useful grid-point updates per second of the exact Eikonal solve.

One step = one pass of the whole hot path over one batch of synthetic input:
per-cell constants c = fl(fl(h/v)^2) and t = +inf, source seeding, and the
persistent bucket-scheduled relaxation to the exact fixed point (Algorithm 6
with the exactly monotone d-bar of arXiv 2103.05694); for the tomography
workload the step adds the adjoint gradient.  Workloads (synthetic, seeded):

  layered_2d     2D layered seismic-like section 2301 x 751, h = 4 m, one
                 surface source (it stands in for the Marmousi section)
  const_2d       2D 129 x 129, constant speed, h = 1/128, centre source
  checker_3d     3D 256^3 smooth random 1500-4500 m/s with a 10:1 checkerboard
                 in the central 128^3 block, h = 10 m, source at (128, 128, 0)
  batched_3d     64 single-source solves on one shared smooth 128^3 model plus
                 24 grids of uneven size (64^3..192^3, 1-4 sources each), one
                 plan replayed from a captured CUDA graph, options autotuned
                 before the timed region (default: the largest single-GPU
                 workload)
  tomography_2d  2D 1024^2, 32 surface sources, 512 receivers: batched forward
                 solve + adjoint gradient of the receiver misfit

Prints one JSON line (rank 0).  Arms:
  default          the CUDA library through its C ABI, inputs resident in HBM;
  --impl reference the CPU oracle (single-threaded fast marching, Algorithm 2,
                   plus the oracle adjoint for tomography) on the host cores,
                   on bounded samples of the same workload.
Multi-GPU (torchrun): the batch and the tomography sources shard by problem
(rank r takes problems r, r + N, ...; strong scaling, no exchange during the
solve; the tomography gradient is gathered on rank 0 and summed in source
order).  A single grid does not shard: every rank solves its own replica
(weak scaling); no collective touches its data.
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
B_ALG = 24          # algorithmic bytes per useful update: read c once, read t once, write t once
L2_FLUSH_BYTES = 512 << 20
# ncu DRAM bytes (read + write) per launch of the persistent kernel in its default
# configuration (the instantiation the timed steps run), from the one-pass
# captures summarised in profiles/ (refresh them whenever the kernel changes)
MEASURED_TRAFFIC = {"layered_2d": 28089088 + 668416, "checker_3d": 283825920 + 117156352}
# ncu DRAM bytes of one launch of the 88-problem batch in the default options
# (the benchmark autotunes, so this is context, not the traffic of the timed launch)
BATCH_TRAFFIC_DEFAULT_OPTIONS = 16199321088 + 2499080704

# FP64 thread instructions (DADD + DMUL + DFMA, ncu sass counters) per operator
# evaluation of the persistent kernel, by dimension, from one-launch captures of
# the counting instantiation (whose evaluation count comes from the same launch;
# the timed instantiation runs the same d-bar code), summarised in profiles/
# (refresh them whenever the kernel changes)
MEASURED_FP64_PER_EVAL = {2: 8.031, 3: 12.982, "batched_3d": 12.717}

WORKLOADS = {
    "layered_2d": "2d_2301x751_layered_h4_1src",
    "const_2d": "2d_129x129_const_h1/128_centre_src",
    "checker_3d": "3d_256cube_smooth_checker_h10_1src",
    "batched_3d": "3d_batch_64x128cube_shared_plus_24_uneven_grids",
    "tomography_2d": "2d_1024x1024_tomography_32src_512rcv_fwd_adj",
}
SINGLE = {"layered_2d": synth.layered_2d_2301x751, "const_2d": synth.const_2d_129,
          "checker_3d": synth.checker_3d_256}


def scaled_layered(scale: float):
    """The layered 2D model at a fraction of its extent per axis (profiling cases)."""
    nx, nz = max(32, round(2301 * scale)), max(8, round(751 * scale))
    speed = synth.layered_section(nx, nz, 4.0, seed=2)
    src = np.array([nx // 2], dtype=np.int64)
    return synth.Problem(f"2d_{nx}x{nz}_layered", speed, 4.0, src, np.zeros(1), {})


def single_problem(args):
    """The single-grid workload, or a reduced case of it (--scale: fraction of
    the extent per axis; layered 2D section and 3D checkerboard volume)."""
    if args.scale != 1.0:
        if args.workload == "layered_2d":
            return scaled_layered(args.scale)
        if args.workload == "checker_3d":
            return synth.checker_3d(max(32, round(256 * args.scale)))
        raise SystemExit("--scale applies to layered_2d and checker_3d")
    return SINGLE[args.workload]()


def useful_of(prob) -> int:
    """Cells the solve must settle: every cell is reachable (speeds > 0), the
    distinct sources are set, not updated."""
    return int(prob.ncells - len(np.unique(prob.sources)))


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
        self.lines = []

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


# --------------------------------------------------------------------------
# CPU oracle legs (reference arm and cpu_baseline)
# --------------------------------------------------------------------------

def oracle_units(args):
    """A list of (label, callable returning useful updates) units of CPU work that
    sample the workload: one full oracle solve (plus adjoint) per unit."""
    import oracle
    oracle.build()
    wl = args.workload
    if wl in SINGLE:
        prob = single_problem(args)

        def unit(p=prob):
            oracle.fmm(p.speed, p.h, p.sources, p.src_t)
            return useful_of(p), 0.0
        return [("full single-threaded FMM solve of the workload", unit)]
    if wl == "batched_3d":
        units = []
        for p in synth.batched_3d():
            def unit(p=p):
                oracle.fmm(p.speed, p.h, p.sources, p.src_t)
                return useful_of(p), 0.0
            units.append((f"FMM solve of problem {p.name}", unit))
        return units
    cfg = synth.tomography_2d_1024()
    h, rcv = cfg["h"], cfg["receivers"]
    v0 = 1.0 / (1.0 / cfg["start"])
    observed = {}
    units = []
    for k, s in enumerate(cfg["sources"]):
        def unit(s=int(s)):
            untimed = 0.0
            if s not in observed:                  # observed data: input, not timed
                t0 = time.perf_counter()
                observed[s] = oracle.fmm(cfg["true"], h, [s]).t
                untimed = time.perf_counter() - t0
            t = oracle.fmm(v0, h, [s]).t
            g = np.zeros(v0.shape)
            g.reshape(-1)[rcv] = (t - observed[s]).reshape(-1)[rcv]
            oracle.adjoint(v0, h, [s], t, g)
            return int(v0.size - 1), untimed
        units.append((f"FMM solve + adjoint of source {k}", unit))
    return units


def time_oracle(units, seconds: float, max_units: int | None = None):
    """Runs units round robin until `seconds` of CPU work (at least one unit)."""
    done, useful, t_sum = 0, 0, 0.0
    per = []
    while True:
        _, fn = units[done % len(units)]
        t0 = time.perf_counter()
        u, untimed = fn()
        dt = time.perf_counter() - t0 - untimed
        per.append(dt)
        useful += u
        t_sum += dt
        done += 1
        if t_sum > seconds or (max_units is not None and done >= max_units):
            break
    return useful, t_sum, per


def run_reference(args, wl_name):
    """The CPU oracle, as it stands, on bounded samples of the same workload."""
    if args.rank != 0:
        return
    units = oracle_units(args)
    if args.warmup > 0:
        units[0][1]()
        if len(units) > 1:
            units = units[1:] + units[:1]
    useful, total, per = time_oracle(units, args.ref_seconds, args.steps)
    value = useful / total
    sample = (f"{len(per)} steps, each one unit of the workload ({units[0][0]}"
              f"{' ...' if len(units) > 1 else ''}), stopping after {args.ref_seconds:.0f} s")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": len(per), "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(per), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl_name},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(args):
    units = oracle_units(args)
    useful, total, per = time_oracle(units, args.cpu_seconds)
    return {"value": useful / total, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(per)} single-threaded oracle units of the workload "
                      f"({units[0][0]}{' ...' if len(units) > 1 else ''}; "
                      f"{total:.1f} s of CPU time on one host core)",
            "ms_per_unit": 1e3 * total / len(per)}


def _oracle_core_worker(workload, items, barrier, out):
    """One host core of the all-cores oracle run: prepares its problems (not
    timed), meets the others at `barrier`, solves its items one by one and
    reports (useful updates, seconds)."""
    import oracle
    work = []
    if workload == "batched_3d":
        model = synth.smooth_model_3d_128()
        for i in items:
            work.append(("fmm", synth.batched_3d_item(i, model)))
    else:
        cfg = synth.tomography_2d_1024()
        h, rcv = cfg["h"], cfg["receivers"]
        v0 = 1.0 / (1.0 / cfg["start"])
        for i in items:
            s = int(cfg["sources"][i])
            observed = oracle.fmm(cfg["true"], h, [s]).t     # the observed data is input
            work.append(("tomo", (v0, h, s, rcv, observed)))
    barrier.wait(timeout=600)       # a worker that failed to start breaks the barrier
    t0 = time.perf_counter()
    useful = 0
    for kind, w in work:
        if kind == "fmm":
            oracle.fmm(w.speed, w.h, w.sources, w.src_t)
            useful += useful_of(w)
        else:
            v0, h, s, rcv, observed = w
            t = oracle.fmm(v0, h, [s]).t
            g = np.zeros(v0.shape)
            g.reshape(-1)[rcv] = (t - observed).reshape(-1)[rcv]
            oracle.adjoint(v0, h, [s], t, g)
            useful += int(v0.size - 1)
    out.put((useful, time.perf_counter() - t0))


def cpu_baseline_all_cores(args, per_unit_s: float, seconds: float = 12.0):
    """The batched and tomography oracle runs as independent solves spread over
    every host core (one process per core, static round-robin assignment,
    started together): the fair batched CPU baseline.  Bounded to about
    `seconds` of work per core; the time is the slowest core's."""
    import multiprocessing as mp
    import oracle
    oracle.build()                                   # once, before the workers load it
    cores = len(os.sched_getaffinity(0))
    n_items = 88 if args.workload == "batched_3d" else 32
    per_core = max(1, min(int(seconds / max(per_unit_s, 1e-3)), -(-n_items // cores)))
    assign = [[(j + cores * k) % n_items for k in range(per_core)] for j in range(cores)]
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_core_worker, args=(args.workload, a, barrier, out))
             for a in assign]
    for pr in procs:
        pr.start()
    try:
        res = [out.get(timeout=900 + 20 * seconds) for _ in procs]
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.terminate()
    useful = sum(u for u, _ in res)
    wall = max(t for _, t in res)
    return {"value": useful / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores * per_core} independent oracle units "
                      f"({'FMM solves of the batch problems' if args.workload == 'batched_3d' else 'FMM solve + adjoint per source'}), "
                      f"{per_core} per process on {cores} host cores, started together; "
                      f"time of the slowest ({wall:.1f} s)"}


# --------------------------------------------------------------------------
# Multi-rank timing (replicas: every rank solves its own copy; the only
# collectives are the timing barrier and the max over ranks)
# --------------------------------------------------------------------------

def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of every rank's x (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, n_ranks: int, total_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank processes the same units)."""
    return units_per_rank * n_ranks / (total_ms / 1e3)


# --------------------------------------------------------------------------
# GPU arms
# --------------------------------------------------------------------------

class Ctx:
    def __init__(self, args):
        import torch
        import paper_2103_05694_gb300 as eik
        from paper_2103_05694_gb300 import build as eikbuild
        eikbuild.build()
        eik.load_library()
        self.torch, self.eik = torch, eik
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local_rank)
        self.local_rank = local_rank
        self.dev = torch.device("cuda", local_rank)
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=self.dev)
            self.dist = dist
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=self.dev)
        self.stream = torch.cuda.current_stream(self.dev)

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        self.torch.cuda.synchronize(self.dev)

    def max_over_ranks(self, x: float) -> float:
        return max_over_ranks(x, self.dist, self.dev)

    def timed(self, steps: int, step_fn):
        """Events around each step on the launching stream, L2 flushed between
        steps outside the events; clocks sampled meanwhile."""
        torch = self.torch
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        self.barrier()
        l0 = self.eik.eik_kernel_launches()
        with ClockSampler(self.local_rank) as clk:
            for i in range(steps):
                evs[i][0].record(self.stream)
                step_fn()
                evs[i][1].record(self.stream)
                self.flush.zero_()
            torch.cuda.synchronize(self.dev)
        launches = self.eik.eik_kernel_launches() - l0
        step_ms = [a.elapsed_time(b) for a, b in evs]
        total = self.max_over_ranks(sum(step_ms))
        self.barrier()
        return total, step_ms, launches, clk.summary()


def time_e2e(C, call, steps):
    torch = C.torch
    for _ in range(2):
        call()
    torch.cuda.synchronize(C.dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(C.stream)
    for _ in range(steps):
        call()
    e1.record(C.stream)
    torch.cuda.synchronize(C.dev)
    return e0.elapsed_time(e1) / steps


def roofline(useful_per_launch: int, kern_ms: float, traffic, what: str):
    peak, kind = measured_peaks()
    achieved = B_ALG * useful_per_launch / (kern_ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": what,
            "kernel_ms": kern_ms, "bytes_per_launch": B_ALG * useful_per_launch,
            "peak_kind": f"{kind} copy bandwidth"}


def roofline_fp64(C, evals_per_launch: int, kern_ms: float, ndim: int, what: str,
                  workload: str | None = None):
    """The FP64 roofline of the persistent kernel: FP64 thread instructions per
    launch (ncu instructions per evaluation x the live evaluation count) over the
    kernel's event time, against the device's measured FP64 add rate."""
    per_eval = MEASURED_FP64_PER_EVAL.get(workload, MEASURED_FP64_PER_EVAL.get(ndim))
    peak = C.eik.eik_fp64_rate() / 1e9
    if per_eval is None:
        return {"bound": "fp64", "achieved": None, "peak": peak, "unit": "G FP64 inst/s",
                "frac": None, "kernel": what, "note": "FP64 instructions per evaluation not "
                "measured for this build", "peak_kind": "measured (eik_fp64_rate, DADD chains)"}
    achieved = per_eval * evals_per_launch / (kern_ms / 1e3) / 1e9
    return {"bound": "fp64", "achieved": achieved, "peak": peak, "unit": "G FP64 inst/s",
            "frac": achieved / peak, "kernel": what, "kernel_ms": kern_ms,
            "fp64_inst_per_eval": per_eval, "evals_per_launch": int(evals_per_launch),
            "peak_kind": "measured (eik_fp64_rate, DADD chains)"}


def base_line(args, n, wl_name, value, total_ms, extra_cfg):
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": n, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict({"workload": wl_name, "parallelism": f"replicas x{n}",
                        "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)"},
                       **extra_cfg),
    }


def make_opts(args):
    opts = {}
    if args.k_delta > 0:
        opts["k_delta"] = args.k_delta
    if args.ctas_per_sm > 0:
        opts["ctas_per_sm"] = args.ctas_per_sm
    if args.window > 0:
        opts["window"] = args.window
    if args.band > 0:
        opts["band"] = args.band
    if args.tile > 0:
        opts["tile"] = args.tile
    if args.update > 0:
        opts["update"] = args.update
    if args.track_changes:
        from paper_2103_05694_gb300 import TRACK_CHANGES
        opts["sched_flags"] = opts.get("sched_flags", 0) | TRACK_CHANGES
    if args.schedule > 0:
        opts["schedule"] = args.schedule
    return opts


def autotuned(args, C, problems, opts):
    """Options from eik_autotune on the timed problems (outside the timed region)."""
    if not args.autotune:
        return opts, None
    t0 = time.perf_counter()
    best, trials = C.eik.eik_autotune(problems, base=opts or None, repeats=1 if len(problems) > 8 else 2)
    info = {"trials": len(trials), "seconds": round(time.perf_counter() - t0, 1),
            "start_ms": trials[0]["ms"], "best_ms": min(t["ms"] for t in trials if t["ms"] > 0)}
    return best, info


def run_single(args, C, wl_name):
    torch, eik = C.torch, C.eik
    prob = single_problem(args)
    if args.scale != 1.0:
        wl_name = prob.name + "_scaled"
    if args.upsample > 1:
        if prob.speed.ndim != 2:
            raise SystemExit("--upsample applies to the 2D workloads")
        prob = synth.upsampled(prob, args.upsample)
        wl_name = f"{wl_name}_upsampled_x{args.upsample}"
    useful = useful_of(prob)
    opts = make_opts(args)
    speed = torch.from_numpy(prob.speed).to(C.dev)
    src = torch.from_numpy(prob.sources).to(C.dev)
    out = torch.empty_like(speed)
    opts, tune = autotuned(args, C, [{"speed": speed, "h": prob.h, "sources": src, "out": out}],
                           opts)

    # correctness gate on the timed configuration: the exact fixed point is reached
    st = eik.solve(speed, prob.h, src, out=out, opts=dict(opts, counters=1)).stats
    torch.cuda.synchronize(C.dev)
    assert st["good"] == useful, (st, useful)
    ref = out.clone()

    for _ in range(args.warmup):
        eik.solve(speed, prob.h, src, out=out, opts=opts)
        C.flush.zero_()
    solve_ms = []

    def step():
        solve_ms.append(eik.solve(speed, prob.h, src, out=out, opts=opts).stats["solve_ms"])
    total_ms, _, launches, clocks = C.timed(args.steps, step)
    same_bits = bool(torch.equal(out, ref))
    assert same_bits or args.update != 0      # d-bar: the same bits on every run (Theorem 1)
    n = args.gpus
    value = job_value(useful * args.steps, n, total_ms)

    # end to end through the C ABI with host buffers (copies inside the call)
    h_speed = torch.from_numpy(prob.speed).pin_memory()
    h_out = torch.empty(prob.speed.shape, dtype=torch.float64).pin_memory()
    h_src = prob.sources.copy()

    def e2e_call():
        if args.schedule:     # device pointers only: copies around the call
            speed.copy_(h_speed, non_blocking=True)
            eik.solve(speed, prob.h, src, out=out, opts=opts)
            h_out.copy_(out, non_blocking=True)
            return
        eik.eik_solve(h_speed.data_ptr(), prob.h, prob.speed.ndim, prob.speed.shape,
                      h_src.ctypes.data, None, len(h_src), h_out.data_ptr(), opts or None,
                      C.stream.cuda_stream)
    e2e_ms = time_e2e(C, e2e_call, max(3, min(args.steps, 30)))
    assert args.update != 0 or np.array_equal(h_out.numpy(), ref.cpu().numpy())
    # Table 3: residual of the computed field under the update that produced it
    bad, max_rel = eik.eik_residual({"speed": speed, "h": prob.h, "sources": src, "out": out},
                                    args.update)

    line = base_line(args, n, wl_name, value, total_ms,
                     {"cells": prob.ncells, "h": prob.h, "sources": int(len(prob.sources)),
                      "opts": opts, "autotune": tune})
    line["grid_point_updates_per_s"] = st["evals"] * args.steps * n / (total_ms / 1e3)
    line["work_per_step"] = {k: st[k] for k in ("evals", "decreases", "good", "visits", "pushes",
                                                "stale_pops", "rounds")}
    line["work_per_step"].update(empty=st["evals"] - st["decreases"],
                                 bad=st["decreases"] - st["good"])
    line["residual"] = {"update": ["d-bar", "d-tilde", "d-hat", "d-hat+Newton"][args.update]
                        + (" (change tracking)" if args.track_changes else ""), "cells": bad,
                        "max_rel": max_rel, "same_bits_every_step": same_bits}
    traffic = args.traffic_bytes
    if traffic is None and not opts and args.scale == 1.0 and args.upsample == 1 and not args.autotune:
        traffic = MEASURED_TRAFFIC.get(args.workload)
    line["roofline"] = roofline(useful, statistics.mean(solve_ms), traffic,
                                ["persistent_kernel (tile relaxation + bucket scheduler)",
                                 "fim_kernel (Algorithm 3 rounds)",
                                 "topo_kernel (Algorithm 4 iterations)",
                                 "fsm_kernel (Algorithm 5 sweeps)"][args.schedule])
    if args.schedule == 0:
        line["roofline_fp64"] = roofline_fp64(C, st["evals"], statistics.mean(solve_ms),
                                              prob.speed.ndim, line["roofline"]["kernel"],
                                              args.workload)
    line["e2e"] = {"value": useful * n / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                   "h2d_bytes_per_step": int(prob.speed.nbytes + h_src.nbytes),
                   "d2h_bytes_per_step": int(prob.speed.nbytes)}
    line["gpu_launches"] = int(launches)
    line["clocks"] = clocks
    return line


def _total_over_ranks(C, x: float) -> float:
    """Sum of x over the ranks (bookkeeping of shard sizes; x itself at N = 1)."""
    if C.dist is None:
        return x
    t = C.torch.tensor([x], device=C.dev, dtype=C.torch.float64)
    C.dist.all_reduce(t)
    return float(t.item())


def run_batched(args, C, wl_name):
    """The 88-problem 3D batch in one persistent launch (a plan replayed from a
    captured CUDA graph).  With N ranks, rank r solves problems r, r + N, ...
    (sharded by problem, no exchange: total work fixed, strong scaling)."""
    from paper_2103_05694_gb300 import shard
    torch, eik = C.torch, C.eik
    n = args.gpus
    n_all = args.problems if args.problems > 0 else 88
    if args.problems > 0:
        wl_name = f"{wl_name}_first{n_all}"
    mine = shard.problem_shard(n_all, args.rank, n)
    model = synth.smooth_model_3d_128()
    probs = [synth.batched_3d_item(i, model) for i in mine]
    useful_mine = sum(useful_of(p) for p in probs)
    useful_all = _total_over_ranks(C, useful_mine)
    opts = make_opts(args)
    dev_speed = {}
    problems = []
    for p in probs:
        key = id(p.speed)
        if key not in dev_speed:
            dev_speed[key] = torch.from_numpy(p.speed).to(C.dev)
        sp = dev_speed[key]
        problems.append({"speed": sp, "h": p.h, "sources": torch.from_numpy(p.sources).to(C.dev),
                         "out": torch.empty_like(sp)})
    opts, tune = autotuned(args, C, problems, opts)
    st = eik.eik_solve_batched(problems, dict(opts, counters=1))
    torch.cuda.synchronize(C.dev)
    assert st["good"] == useful_mine, (st["good"], useful_mine)
    refs = [q["out"].clone() for q in problems]

    # kernel-only duration of the persistent launch (events inside the library)
    solve_ms = [eik.eik_solve_batched(problems, opts)["solve_ms"] for _ in range(3)]

    plan = eik.Plan([dict(q) for q in problems], opts)
    side = torch.cuda.Stream(C.dev)
    side.wait_stream(C.stream)
    plan.enqueue(side)
    plan.status(side)
    graph = torch.cuda.CUDAGraph()
    l0 = eik.eik_kernel_launches()
    with torch.cuda.graph(graph, stream=side):
        plan.enqueue(side)
    per_replay = eik.eik_kernel_launches() - l0
    for _ in range(args.warmup):
        graph.replay()
        C.flush.zero_()
    torch.cuda.synchronize(C.dev)
    total_ms, _, _, clocks = C.timed(args.steps, graph.replay)
    plan.status(C.stream)                  # raises unless the last replay succeeded
    for q, r in zip(problems, refs):
        assert torch.equal(q["out"], r)
    value = useful_all * args.steps / (total_ms / 1e3)

    # end to end through the C ABI: one eik_solve_batched call per step on
    # pinned host buffers (the call stages the models in, solves, and copies
    # every field back)
    h_speed = {}
    for p in probs:
        if id(p.speed) not in h_speed:
            h_speed[id(p.speed)] = torch.from_numpy(p.speed).pin_memory()
    host_problems = [{"speed": h_speed[id(p.speed)], "h": p.h,
                      "sources": np.ascontiguousarray(p.sources, dtype=np.int64),
                      "out": torch.empty(p.speed.shape, dtype=torch.float64).pin_memory()}
                     for p in probs]

    e2e_retries = []

    def e2e_call():
        e2e_retries.append(eik.eik_solve_batched(host_problems, opts, C.stream)["retries"])
    e2e_ms = time_e2e(C, e2e_call, 3)
    for hp, r in zip(host_problems, refs):
        assert np.array_equal(hp["out"].numpy(), r.cpu().numpy())
    h2d = sum(t.numel() * 8 for t in h_speed.values()) + sum(p.sources.nbytes for p in probs)
    d2h = sum(p.speed.nbytes for p in probs)
    e2e_ms = C.max_over_ranks(e2e_ms)

    line = base_line(args, n, wl_name, value, total_ms,
                     {"problems": n_all, "problems_per_rank": len(probs),
                      "cells": int(_total_over_ranks(C, sum(p.ncells for p in probs))),
                      "distinct_models": len(dev_speed), "captured_graph": True, "opts": opts,
                      "autotune": tune})
    if n > 1:
        line["scaling"] = "strong"
        line["config"]["parallelism"] = f"sharded by problem x{n} (rank r: problems r, r+{n}, ...)"
    line["work_per_step"] = {k: st[k] for k in ("evals", "decreases", "good", "visits", "pushes",
                                                "stale_pops", "rounds")}
    line["work_per_step"].update(empty=st["evals"] - st["decreases"],
                                 bad=st["decreases"] - st["good"])
    line["roofline"] = roofline(useful_mine, statistics.mean(solve_ms), args.traffic_bytes,
                                "persistent_kernel (all problems in one launch)")
    if args.problems == 0:
        line["roofline"]["traffic_default_options"] = BATCH_TRAFFIC_DEFAULT_OPTIONS
    line["roofline_fp64"] = roofline_fp64(C, st["evals"], statistics.mean(solve_ms), 3,
                                          line["roofline"]["kernel"], "batched_3d")
    line["e2e"] = {"value": useful_all / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "call": "eik_solve_batched with pinned host buffers (read and written in place by the library's kernels inside the call)",
                   "capacity_retries": int(sum(e2e_retries))}
    line["gpu_launches"] = int(per_replay * args.steps)
    line["clocks"] = clocks
    plan.close()
    return line


def run_tomography(args, C, wl_name):
    """Batched forward + adjoint gradient of the receiver misfit.  At N = 1 the
    step is the differentiable solve (eikonal + autograd); with N ranks, rank r
    solves sources r, r + N, ... and its per-source gradients are gathered on
    rank 0, which sums them in source order (bit-identical to N = 1)."""
    from paper_2103_05694_gb300 import shard
    torch, eik = C.torch, C.eik
    cfg = synth.tomography_2d_1024()
    h = cfg["h"]
    sources = cfg["sources"][:args.sources] if args.sources > 0 else cfg["sources"]
    n_src = len(sources)
    n = args.gpus
    mine = shard.problem_shard(n_src, args.rank, n)
    s0 = torch.from_numpy(1.0 / cfg["start"]).to(C.dev)
    srcs = [torch.tensor([int(sources[i])], device=C.dev) for i in mine]
    rcv = torch.from_numpy(cfg["receivers"]).to(C.dev)
    with torch.no_grad():
        t_obs = eik.eikonal(torch.from_numpy(1.0 / cfg["true"]).to(C.dev), h, srcs) \
            .reshape(len(srcs), -1)[:, rcv].contiguous()
    useful_all = n_src * (s0.numel() - 1)

    def grad_of(s_dev):
        s = s_dev.detach().requires_grad_(True)
        t = eik.eikonal(s, h, srcs)
        loss = 0.5 * ((t.reshape(len(srcs), -1)[:, rcv] - t_obs) ** 2).sum()
        loss.backward()
        return s.grad

    # sharded step: per-source gradients (no sum) -> gather -> ordered sum on rank 0
    outs = torch.empty((len(srcs),) + tuple(s0.shape), dtype=torch.float64, device=C.dev)
    gts = torch.zeros_like(outs)
    grads = torch.empty_like(outs)
    g_total = torch.empty_like(s0)

    def grad_sharded(s_dev):
        probs = [{"speed": s_dev, "h": h, "sources": src, "out": outs[i]} for i, src in enumerate(srcs)]
        eik.eik_solve_batched(probs, {"sched_flags": eik.SLOWNESS_INPUT})
        gts.reshape(len(srcs), -1)[:, rcv] = outs.reshape(len(srcs), -1)[:, rcv] - t_obs
        eik.eik_adjoint(probs, [gts[i] for i in range(len(srcs))], [grads[i] for i in range(len(srcs))],
                        {"sched_flags": eik.SLOWNESS_INPUT})
        allg = shard.gather_items(grads, n_src, args.rank, n, C.dist, dst=0)
        if allg is not None:
            eik.eik_sum_ordered([allg[i] for i in range(n_src)], g_total)
        return g_total

    step = grad_of if n == 1 else grad_sharded
    g_ref = step(s0).clone()
    for _ in range(args.warmup):
        step(s0)
        C.flush.zero_()
    torch.cuda.synchronize(C.dev)
    total_ms, _, launches, clocks = C.timed(args.steps, lambda: step(s0))
    g_last = step(s0)
    if args.rank == 0:
        assert torch.equal(g_last, g_ref)       # the gradient is deterministic
    value = useful_all * args.steps / (total_ms / 1e3)

    per_source_ms = None
    if n == 1:
        # the same gradient from per-source solves and adjoints (one problem per call)
        speed = torch.reciprocal(s0)
        po = [torch.empty_like(s0) for _ in srcs]
        pg = [torch.empty_like(s0) for _ in srcs]

        def per_source():
            total = torch.zeros_like(s0)
            for i, src in enumerate(srcs):
                eik.solve(speed, h, src, out=po[i])
                gt = torch.zeros_like(s0)
                gt.reshape(-1)[rcv] = po[i].reshape(-1)[rcv] - t_obs[i]
                eik.eik_adjoint([{"speed": speed, "h": h, "sources": src, "out": po[i]}], [gt],
                                [pg[i]])
                total += pg[i]
            return total
        g_ps = per_source()
        torch.cuda.synchronize(C.dev)
        assert torch.allclose(g_ps, g_ref, rtol=1e-12, atol=1e-12 * float(g_ref.abs().max()))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, 3))
        e0.record(C.stream)
        for _ in range(reps):
            per_source()
        e1.record(C.stream)
        torch.cuda.synchronize(C.dev)
        per_source_ms = e0.elapsed_time(e1) / reps

    # kernel-only duration of the batched forward launch
    probs = [{"speed": s0, "h": h, "sources": src, "out": outs[i]} for i, src in enumerate(srcs)]
    fwd_evals = eik.eik_solve_batched(probs, {"sched_flags": eik.SLOWNESS_INPUT, "counters": 1})["evals"]
    solve_ms = [eik.eik_solve_batched(probs, {"sched_flags": eik.SLOWNESS_INPUT})["solve_ms"]
                for _ in range(3)]

    # end to end: slowness from pinned host memory, gradient back to the host
    h_s = s0.cpu().pin_memory()
    h_g = torch.empty_like(h_s).pin_memory()

    def e2e_call():
        g = step(h_s.to(C.dev, non_blocking=True))
        if args.rank == 0:
            h_g.copy_(g, non_blocking=True)
    e2e_ms = C.max_over_ranks(time_e2e(C, e2e_call, max(3, min(args.steps, 10))))
    if args.rank == 0:
        assert torch.equal(h_g, g_ref.cpu())

    line = base_line(args, n, wl_name, value, total_ms,
                     {"cells": int(s0.numel()), "h": h, "sources": n_src,
                      "receivers": int(rcv.numel()), "step": "batched forward + adjoint + misfit"})
    if n > 1:
        line["scaling"] = "strong"
        line["config"]["parallelism"] = (f"sharded by source x{n}; per-source gradients gathered "
                                         "on rank 0 and summed in source order")
    line["tomography"] = {"batched_step_ms": total_ms / args.steps,
                          "per_source_step_ms": per_source_ms,
                          "speedup_vs_per_source": (per_source_ms / (total_ms / args.steps)
                                                    if per_source_ms else None)}
    line["roofline"] = roofline(len(srcs) * (s0.numel() - 1), statistics.mean(solve_ms),
                                args.traffic_bytes, "persistent_kernel (batched forward)")
    line["roofline_fp64"] = roofline_fp64(C, fwd_evals, statistics.mean(solve_ms), 2,
                                          line["roofline"]["kernel"])
    line["e2e"] = {"value": useful_all / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                   "h2d_bytes_per_step": int(h_s.numel() * 8),
                   "d2h_bytes_per_step": int(h_g.numel() * 8)}
    line["gpu_launches"] = int(launches)
    line["clocks"] = clocks
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_3d", choices=sorted(WORKLOADS))
    ap.add_argument("--scale", type=float, default=1.0,
                    help="layered_2d and checker_3d: fraction of the extent per axis (profiling)")
    ap.add_argument("--upsample", type=int, default=1,
                    help="2D single grids: nearest-neighbour upsampling by this factor per axis, "
                         "spacing h / factor (Table 3's input scale)")
    ap.add_argument("--problems", type=int, default=0,
                    help="batched_3d only: the first N of the 88 problems (profiling cases; "
                         "no CPU baseline); 0: all")
    ap.add_argument("--sources", type=int, default=0,
                    help="tomography_2d only: use the first N sources (profiling cases)")
    ap.add_argument("--k-delta", type=float, default=0.0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--band", type=float, default=0.0)
    ap.add_argument("--tile", type=int, default=0,
                    help="tile shape 1-5 (see eik_opts.tile); 0: automatic")
    ap.add_argument("--schedule", type=int, default=0,
                    help="single grids: 1 = fast iterative method (Algorithm 3), 2 = "
                         "topology-driven (Algorithm 4), 3 = fast sweeping (Algorithm 5); "
                         "0: asynchronous tiles (Algorithm 6)")
    ap.add_argument("--update", type=int, default=0,
                    help="2D ablation: 1 = Algorithm 1 with d-tilde, 2 = with d-hat, 3 = d-hat "
                         "then Newton (0: d-bar)")
    ap.add_argument("--track-changes", action="store_true",
                    help="with --update 1-3: conservative work tracking (activate on any change)")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=None,
                    help="pick the scheduling options with eik_autotune on the workload first "
                         "(outside the timed region); default: on for batched_3d")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="ncu dram bytes per launch of the solve kernel, if measured")
    args = ap.parse_args()
    if args.problems and (args.workload != "batched_3d" or not 0 < args.problems <= 88):
        raise SystemExit("--problems takes 1..88 and applies to batched_3d only")
    args.rank = int(os.environ.get("RANK", "0"))
    if args.autotune is None:
        args.autotune = args.workload == "batched_3d"
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        args.gpus = world
    wl_name = WORKLOADS[args.workload]
    if args.workload == "tomography_2d" and args.sources > 0:
        wl_name = wl_name.replace("32src", f"{args.sources}src")

    if args.impl == "reference":
        run_reference(args, wl_name)
        return

    C = Ctx(args)
    if args.workload in SINGLE:
        line = run_single(args, C, wl_name)
    elif args.workload == "batched_3d":
        line = run_batched(args, C, wl_name)
    else:
        line = run_tomography(args, C, wl_name)
    if args.rank == 0 and args.gpus == 1 and not args.no_cpu_baseline and args.problems == 0:
        line["cpu_baseline"] = cpu_baseline(args)
        if args.workload in ("batched_3d", "tomography_2d"):
            line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(
                args, line["cpu_baseline"]["ms_per_unit"] / 1e3, args.cpu_seconds)
    if args.rank == 0:
        print(json.dumps(line), flush=True)
    if C.dist is not None:
        C.dist.destroy_process_group()


if __name__ == "__main__":
    main()

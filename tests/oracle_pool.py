"""Oracle solves of the full-size workloads spread over the host cores.

Each job names one problem of a workload; a spawned worker process (spawn,
never fork: the parent holds a CUDA context) regenerates it from its seed with
`synth`, solves it with the CPU oracle and returns the SHA-256 of the arrival
times' bytes (and, for tomography sources, the oracle adjoint gradient), so
that every problem can be compared with the GPU result bit for bit without
shipping the fields between processes.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

_MODEL = None
_TOMO = None


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float64).tobytes()).hexdigest()


def _job(job):
    import oracle
    import synth
    global _MODEL, _TOMO
    kind, i = job
    if kind == "batch":
        if _MODEL is None:
            _MODEL = synth.smooth_model_3d_128()
        p = synth.batched_3d_item(i, _MODEL)
        return job, (digest(oracle.fmm(p.speed, p.h, p.sources, p.src_t).t),), None
    if _TOMO is None:
        cfg = synth.tomography_2d_1024()
        _TOMO = (cfg, 1.0 / (1.0 / cfg["start"]))
    cfg, v = _TOMO
    h, rcv = cfg["h"], cfg["receivers"]
    s = int(cfg["sources"][i])
    t = oracle.fmm(v, h, [s]).t
    t_obs = oracle.fmm(cfg["true"], h, [s]).t
    g = np.zeros(v.shape)
    g.reshape(-1)[rcv] = (t - t_obs).reshape(-1)[rcv]
    return job, (digest(t), digest(t_obs)), oracle.adjoint(v, h, [s], t, g)[1]


def run(jobs, processes: int | None = None) -> dict:
    """{job: (digests, gradient or None)} for jobs ("batch", i) / ("tomo", k): the
    digests of the times (and, for a tomography source, of the observed times
    on the true model), and the oracle adjoint gradient of the misfit."""
    import multiprocessing as mp
    import oracle
    oracle.build()                       # once, before the workers load it
    n = processes or max(1, len(os.sched_getaffinity(0)))
    with mp.get_context("spawn").Pool(min(n, len(jobs))) as pool:
        out = {}
        for job, dig, grad in pool.imap_unordered(_job, jobs):
            out[job] = (dig, grad)
    return out

"""Seeded synthetic inputs for the Eikonal solver and its oracle.

This module only draws and shapes speed fields and source sets (numpy PCG64,
fixed seeds).  It holds none of the solver's arithmetic: both the CUDA path and
the CPU oracle take their inputs from here.

The paper's workload is the Elastic Marmousi model, a 2801 x 13601 speed map at
1.25 m spacing, nearest-neighbour upsampled x4 per axis (Methods).  That dataset
is not available here; the generators below stand in for it with seismic-shaped
synthetic models (layered 2D section with faults, smooth random 3D volumes with
a high-contrast checkerboard, batches of uneven grids, a tomography pair).

Arrays are C-order with x (the last axis) contiguous: 2D speed has shape
(nz, nx), 3D has (nz, ny, nx).  Sources are flat C-order cell indices.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.ndimage import gaussian_filter1d


@dataclass
class Problem:
    name: str
    speed: np.ndarray            # float64, shape (nz, nx) or (nz, ny, nx)
    h: float
    sources: np.ndarray          # int64 flat indices
    src_t: np.ndarray            # float64 source times
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.speed.shape

    @property
    def ncells(self) -> int:
        return int(self.speed.size)


def smooth(noise: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian filter truncated at 4 sigma, reflecting boundaries."""
    out = noise
    for ax in range(noise.ndim):
        out = gaussian_filter1d(out, sigma, axis=ax, mode="reflect", truncate=4.0)
    return out


def _flat(shape, *coords) -> int:
    return int(np.ravel_multi_index(tuple(int(c) for c in coords), shape))


def const_2d_129() -> Problem:
    """2D 129 x 129, h = 1/128, constant speed 1, one source at the centre cell."""
    n = 129
    speed = np.ones((n, n), dtype=np.float64)
    src = np.array([_flat((n, n), 64, 64)], dtype=np.int64)
    return Problem("2d_129x129_const", speed, 1.0 / 128.0, src, np.zeros(1),
                   {})


def layered_section(nx: int = 2301, nz: int = 751, h: float = 4.0, seed: int = 2,
                    n_interfaces: int = 12, n_faults: int = 3) -> np.ndarray:
    """Marmousi-like 2D section: sinusoidal layer interfaces, dipping faults
    that shift the hanging wall down, a smooth 5 % multiplicative perturbation,
    clipped to [1500, 5500] m/s.  Shape (nz, nx)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.arange(nx, dtype=np.float64) * h
    z = np.arange(nz, dtype=np.float64) * h
    depth = nz * h
    amp = rng.uniform(20.0, 80.0, n_interfaces)
    lam = rng.uniform(1000.0, 5000.0, n_interfaces)
    phase = rng.uniform(0.0, 2.0 * np.pi, n_interfaces)
    base = np.linspace(0.0, depth, n_interfaces + 2)[1:-1]
    iface = base[:, None] + amp[:, None] * np.sin(2.0 * np.pi * x[None, :] / lam[:, None]
                                                  + phase[:, None])      # (k, nx)
    n_layers = n_interfaces + 1
    layer_v = np.linspace(1500.0, 5500.0, n_layers) * (1.0 + rng.uniform(-0.05, 0.05, n_layers))
    zz = np.broadcast_to(z[:, None], (nz, nx)).copy()                    # effective depth
    xx = np.broadcast_to(x[None, :], (nz, nx))
    for _ in range(n_faults):
        x0 = rng.uniform(0.0, nx * h)
        dip = np.deg2rad(rng.uniform(55.0, 80.0))
        throw = rng.uniform(40.0, 200.0)
        hanging = xx > x0 + z[:, None] / np.tan(dip)
        zz = np.where(hanging, zz - throw, zz)
    layer = np.zeros((nz, nx), dtype=np.int64)
    for k in range(n_interfaces):
        layer += (zz > iface[k][None, :]).astype(np.int64)
    v = layer_v[layer]
    g = smooth(rng.standard_normal((nz, nx)), 5.0)
    g /= g.std()
    v = v * (1.0 + 0.05 * g)
    return np.clip(v, 1500.0, 5500.0)


def layered_2d_2301x751() -> Problem:
    """2D layered seismic-like model 2301 (x) x 751 (z), h = 4 m, one surface
    source at x = 4600 m."""
    h = 4.0
    speed = layered_section(2301, 751, h, seed=2)
    src = np.array([_flat(speed.shape, 0, 1150)], dtype=np.int64)
    return Problem("2d_2301x751_layered", speed, h, src, np.zeros(1), {})


def upsampled(p: Problem, k: int) -> Problem:
    """A 2D problem upsampled by k on each axis with nearest-neighbour
    interpolation (spacing h / k), its sources at the same physical points: the
    paper's x4 input scale (Methods: Marmousi upsampled by 4 per axis)."""
    if k == 1:
        return p
    nz, nx = p.speed.shape
    speed = np.repeat(np.repeat(p.speed, k, axis=0), k, axis=1)
    z, x = np.divmod(p.sources, nx)
    src = (z * k) * (nx * k) + x * k
    return Problem(f"{p.name}_up{k}", speed, p.h / k, src.astype(np.int64), p.src_t.copy(),
                   dict(p.meta, upsample=k))


def smooth_random_volume(n: int, seed: int, vmin: float, vmax: float,
                         sigma: float = 8.0) -> np.ndarray:
    """White noise, Gaussian-filtered, affinely mapped from its min/max to
    [vmin, vmax].  Shape (n, n, n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = smooth(rng.standard_normal((n, n, n)), sigma)
    lo, hi = g.min(), g.max()
    return vmin + (g - lo) * ((vmax - vmin) / (hi - lo))


def checker_3d(n: int = 256) -> Problem:
    """3D n^3, h = 10 m, smooth random 1500-4500 m/s with a 16^3-cell 10:1
    checkerboard (slow cells v/10) in the central (n/2)^3 block; source at
    (x, y, z) = (n/2, n/2, 0).  n = 256 is the benchmark volume; smaller n give
    reduced cases of the same structure (profiling)."""
    v = smooth_random_volume(n, 3, 1500.0, 4500.0, 8.0)
    lo, hi = n // 4, n // 4 + n // 2
    idx = np.arange(lo, hi)
    cz, cy, cx = np.meshgrid(idx // 16, idx // 16, idx // 16, indexing="ij")
    slow = ((cz + cy + cx) % 2) == 1
    block = v[lo:hi, lo:hi, lo:hi]
    v[lo:hi, lo:hi, lo:hi] = np.where(slow, block / 10.0, block)
    src = np.array([_flat(v.shape, 0, n // 2, n // 2)], dtype=np.int64)
    name = "3d_256_checker" if n == 256 else f"3d_{n}_checker"
    return Problem(name, v, 10.0, src, np.zeros(1), {})


def checker_3d_256() -> Problem:
    """3D 256^3, h = 10 m, smooth random 1500-4500 m/s with a 16^3-cell 10:1
    checkerboard (slow cells v/10) in the central 128^3 block; source at
    (x, y, z) = (128, 128, 0)."""
    return checker_3d(256)


def smooth_model_3d_128(n: int = 128) -> np.ndarray:
    return smooth_random_volume(n, 4, 1500.0, 4500.0, 8.0)


def batched_3d_item(i: int, model: np.ndarray | None = None, n_lattice: int = 8,
                    model_n: int = 128) -> Problem:
    """Problem i of batched_3d, generated alone (`model`: the shared lattice
    model, if already at hand)."""
    h = 10.0
    if i < n_lattice * n_lattice:
        if model is None:
            model = smooth_model_3d_128(model_n)
        yy, xx = 8 + 16 * (i // n_lattice), 8 + 16 * (i % n_lattice)
        src = np.array([_flat(model.shape, 0, yy, xx)], dtype=np.int64)
        return Problem(f"shared_src_{yy}_{xx}", model, h, src, np.zeros(1), {"shared_model": True})
    k = i - n_lattice * n_lattice
    rng = np.random.Generator(np.random.PCG64(400 + k))
    side = int(rng.integers(64, 193))
    v = smooth_random_volume(side, 400 + k, 1500.0, 4500.0, 8.0)
    ns = int(rng.integers(1, 5))
    src = np.unique(rng.integers(0, side ** 3, ns)).astype(np.int64)
    return Problem(f"grid_{k}_{side}", v, h, src, np.zeros(src.size), {"shared_model": False})


def batched_3d(n_lattice: int = 8, n_grids: int = 24, model_n: int = 128) -> list[Problem]:
    """Batched multi-source work: one solve per source on a lattice of surface
    sources over a shared smooth 128^3 model, plus independent grids of uneven
    size (side uniform in 64..192, own model, 1-4 sources solved together)."""
    model = smooth_model_3d_128(model_n)
    return [batched_3d_item(i, model, n_lattice, model_n)
            for i in range(n_lattice * n_lattice + n_grids)]


def tomography_2d_1024(n: int = 1024, n_src: int = 32, n_rcv: int = 512, z_c: float | None = None):
    """Tomography pair on a 1024^2 grid, h = 5 m: smooth random background
    2000-4000 m/s (sigma 16 cells); the true model adds a +10 % and a -10 %
    Gaussian anomaly (sigma 60 cells) at 1/3 and 2/3 of the width, centred at
    half the depth that surface first arrivals reach.  That depth is about
    n/16 rows on this background (no depth trend: first arrivals between
    surface points stay within ~45 rows at n = 1024), so z_c defaults to n/32;
    anomalies at half the full depth would change the observed times by about
    1e-13 relative, below the rounding of the times.  Surface sources at
    x = 16 + 32k, receivers at x = 1 + 2k."""
    h = 5.0
    rng = np.random.Generator(np.random.PCG64(5))
    g = smooth(rng.standard_normal((n, n)), 16.0)
    background = 2000.0 + (g - g.min()) * (2000.0 / (g.max() - g.min()))
    zz, xx = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64),
                         indexing="ij")
    sig = 60.0
    zc = n / 32.0 if z_c is None else float(z_c)
    bump1 = np.exp(-(((xx - n / 3.0) ** 2 + (zz - zc) ** 2) / (2.0 * sig * sig)))
    bump2 = np.exp(-(((xx - 2.0 * n / 3.0) ** 2 + (zz - zc) ** 2) / (2.0 * sig * sig)))
    true = background * (1.0 + 0.10 * bump1 - 0.10 * bump2)
    sources = np.array([_flat((n, n), 0, 16 + 32 * k) for k in range(n_src)], dtype=np.int64)
    receivers = np.array([_flat((n, n), 0, 1 + 2 * k) for k in range(n_rcv)], dtype=np.int64)
    return {"h": h, "true": true, "start": background, "sources": sources,
            "receivers": receivers}


def random_problem(seed: int, shape, n_src: int = 1, contrast: float = 10.0,
                   smooth_sigma: float | None = None, h: float = 1.0,
                   src_t_max: float = 0.0) -> Problem:
    """A small random problem: speeds in [1, contrast] (white noise or smoothed),
    n_src distinct random sources with times in [0, src_t_max]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(int(s) for s in shape)
    u = rng.random(shape)
    if smooth_sigma:
        u = smooth(u, smooth_sigma)
        u = (u - u.min()) / max(u.max() - u.min(), 1e-300)
    speed = 1.0 + (contrast - 1.0) * u
    N = int(np.prod(shape))
    n_src = min(n_src, N)
    src = rng.choice(N, size=n_src, replace=False).astype(np.int64)
    st = rng.random(n_src) * src_t_max if src_t_max > 0 else np.zeros(n_src)
    return Problem(f"random_{seed}_{'x'.join(map(str, shape))}", speed, h, src, st,
                   {"seed": seed})


def shuffled_order(seed: int, n: int) -> np.ndarray:
    """A random permutation of range(n) (an input for order-independence tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.permutation(n).astype(np.int64)

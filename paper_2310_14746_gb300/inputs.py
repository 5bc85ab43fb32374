"""Seeded synthetic inputs: porosity-control fields, random states, request streams.

This module holds no arithmetic of the lattice scheme itself. It renders
geometry (periodic sphere matrices, Sec. 2.1 of Simonis et al.,
arXiv:2310.14746, Part I) into a per-cell porosity control varpi in [0, 1]
(varpi = 1 free fluid, varpi = 0 solid; eq. "d definition" names the field)
and draws seeded random numbers. Both the CUDA path and the CPU oracle take
these arrays as inputs.

Smoothing of the sphere field (the paper does not discretize geometry): with
s the periodic distance from a cell centre (integer + 1/2) to the nearest
sphere centre minus the radius, varpi = (1 + sin(pi * clamp(s/w, -1/2, 1/2)))/2
with a transition width w of 2 cells.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_WIDTH = 2.0
SEED_BASE = 2310147460


def _smooth_step(s: np.ndarray, width: float) -> np.ndarray:
    t = np.clip(s / width, -0.5, 0.5)
    return 0.5 * (1.0 + np.sin(np.pi * t))


def _shape3(n) -> tuple:
    if np.isscalar(n):
        return (int(n),) * 3
    nx, ny, nz = (int(v) for v in n)
    return nx, ny, nz


def regular_sphere_field(n, period: float = 32.0, radius_ratio: float = 0.3,
                         width: float = DEFAULT_WIDTH, dtype=np.float32) -> np.ndarray:
    """Regular periodic matrix of equal spheres (one per cubic cell of edge `period`,
    centred in it) rendered as a smoothed varpi[z][y][x]. `n` is an edge or (nx, ny, nz)."""
    nx, ny, nz = _shape3(n)
    r = radius_ratio * period

    def axis(m):
        t = np.mod(np.arange(m) + 0.5, period) - 0.5 * period
        return t * t

    d2 = axis(nz)[:, None, None] + axis(ny)[None, :, None] + axis(nx)[None, None, :]
    s = np.sqrt(d2) - r
    return _smooth_step(s, width).astype(dtype)


def sphere_matrix_porosity(radius_ratio: float) -> float:
    """Void fraction of one sphere of radius r = radius_ratio * P per cubic cell of edge P
    (Prop. porosity, with the radius in place of the diameter)."""
    return 1.0 - 4.0 / 3.0 * math.pi * radius_ratio ** 3


def boolean_sphere_geometry(seed: int, phi_target: float, radius: float):
    """Centres (uniform in the unit torus [0,1)^3) of a Boolean model of equal spheres of
    `radius` (a fraction of the box edge), with the count chosen so that the expected void
    fraction exp(-count * 4/3 pi r^3) equals phi_target."""
    rng = np.random.default_rng(seed)
    vol = 4.0 / 3.0 * math.pi * radius ** 3
    count = max(1, int(round(-math.log(phi_target) / vol)))
    return rng.random((count, 3)), radius


def render_sphere_geometry(n, centres: np.ndarray, radius: float,
                           width: float = DEFAULT_WIDTH, dtype=np.float32,
                           slab: int = 16) -> np.ndarray:
    """Render spheres (unit-torus centres, radius as a box fraction) onto an n^3 grid as a
    smoothed varpi field. The same geometry renders at any resolution."""
    from scipy.spatial import cKDTree

    nx, ny, nz = _shape3(n)
    assert nx == ny == nz, "unit-torus geometry renders on cubic grids"
    scaled = np.mod(centres * n, n)
    tree = cKDTree(scaled, boxsize=float(n))
    r = radius * n
    out = np.empty((nz, ny, nx), dtype=dtype)
    yy, xx = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        zz = np.arange(z0, z1) + 0.5
        pts = np.stack([
            np.broadcast_to(xx, (z1 - z0, ny, nx)),
            np.broadcast_to(yy, (z1 - z0, ny, nx)),
            np.broadcast_to(zz[:, None, None], (z1 - z0, ny, nx)),
        ], axis=-1).reshape(-1, 3)
        d, _ = tree.query(np.mod(pts, n), k=1, workers=-1)
        out[z0:z1] = _smooth_step(d - r, width).reshape(z1 - z0, ny, nx).astype(dtype)
    return out


def random_sphere_field(n: int, seed: int, period: float = 32.0,
                        radius_ratio_range=(0.1, 0.45), phi_range=(0.4, 0.9),
                        width: float = DEFAULT_WIDTH, render_n: int | None = None):
    """Random periodic (Boolean) sphere matrix: radius r = period * U[radius_ratio_range]
    (in cells of an n^3 box), target void fraction phi* ~ U[phi_range]; rendered at
    `render_n` (default n) so that a coarser grid samples the same continuous field.
    Returns (varpi, info)."""
    rng = np.random.default_rng(seed)
    ratio = float(rng.uniform(*radius_ratio_range))
    phi = float(rng.uniform(*phi_range))
    radius = ratio * period / n
    centres, radius = boolean_sphere_geometry(seed + 1, phi, radius)
    m = n if render_n is None else render_n
    field = render_sphere_geometry(m, centres, radius, width=width)
    info = {"radius_ratio": ratio, "phi_target": phi, "spheres": int(len(centres)),
            "radius_cells": radius * m}
    return field, info


def random_populations(q: int, shape, seed: int, amplitude: float = 0.5) -> np.ndarray:
    """Random positive populations f[q][...] = (1 + amplitude * U(-1, 1)) / q (float64)."""
    rng = np.random.default_rng(seed)
    return (1.0 + amplitude * rng.uniform(-1.0, 1.0, size=(q,) + tuple(shape))) / q


def random_porosity(shape, seed: int, lo: float = 0.2, hi: float = 1.0,
                    dtype=np.float32) -> np.ndarray:
    """Uniform random varpi in [lo, hi] per cell."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=tuple(shape)).astype(dtype)


SERVING_EDGES = (32, 64, 96, 128, 192)


def serving_requests(n_requests: int, seed: int, rate_per_s: float):
    """Solve requests for the serving stream: Poisson arrivals at `rate_per_s`, lattice edge
    uniform in SERVING_EDGES, sphere period uniform over the divisors of the edge in
    [16, 64] (so the field is periodic on the box), radius ratio ~ U[0.1, 0.45]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s)) if rate_per_s > 0 else 0.0
        edge = int(rng.choice(SERVING_EDGES))
        periods = [p for p in range(16, 65) if edge % p == 0]
        period = int(rng.choice(periods))
        ratio = float(rng.uniform(0.1, 0.45))
        out.append({"id": k, "arrival_s": t, "edge": edge, "period": period,
                    "radius_ratio": ratio})
    return out

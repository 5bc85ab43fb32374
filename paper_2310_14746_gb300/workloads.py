"""Workloads built on the step kernel beyond the forced steady solve.

memory_kernel: the time-dependent permeability of the Darcy law with memory
(Simonis et al., arXiv:2310.14746, Part I, Sec. 2: the unit-cell problem for
A~(t) and A = integral of A~ dt). A periodic cell relaxes from a uniform velocity
u0 e_axis with no force; A~_n = <rho u_axis>_n / u0 is its normalised mean
momentum after n steps, and sum_n A~_n (dt = 1) approximates K / nu, the
apparent permeability of the forced steady problem divided by the viscosity.
For uniform porosity the shift form relaxes as u_n = u0 (1 - lam)^n,
lam = (1 - varpi)/tau, so the sum is exactly 1/lam = tau / (1 - varpi) = K / nu.

permeability_pair: the apparent permeability of one sphere per periodic cell of
edge P, resolved (a voxel sphere with bounce-back on its surface, varpi = 1 in
the fluid: the unit-cell problem of Thm. thmStatNSECase4) and homogenized (the
smoothed varpi field of the same sphere), next to the dilute-array drag
correlation of Hasimoto (1959) with the coefficients of Sangani & Acrivos
(1982), evaluated at the voxel sphere's volume-equivalent radius.
"""
from __future__ import annotations

import math

import numpy as np

from . import HLBM_D3Q19, HLBM_F32, HLBM_TWO_LATTICE, Lattice


def memory_kernel(varpi, tau, steps, u0=1e-4, axis=0, storage=HLBM_F32, pattern=HLBM_TWO_LATTICE,
                  velset=HLBM_D3Q19, stop_below=0.0, chunk=4096):
    """Return A~_n for n = 0..steps-1 (numpy float64), stopping early once |A~_n| < stop_below.
    The mean momentum is recorded on the device after every step (hlbm_reduce_series) and read
    back once per chunk of steps, so the host never waits on a single step."""
    varpi = np.ascontiguousarray(varpi, dtype=np.float32)
    nz, ny, nx = varpi.shape
    cells = nx * ny * nz
    lat = Lattice(velset, nx, ny, nz, storage, pattern)
    try:
        lat.set_relaxation(tau)
        lat.set_force(0.0, 0.0, 0.0)
        lat.set_porosity(varpi)
        u = [0.0, 0.0, 0.0]
        u[axis] = u0
        lat.init_equilibrium(1.0, u)
        col = 1 + axis  # mom_x, mom_y, mom_z
        out = []
        done = 0
        while done < steps:
            m = min(chunk, steps - done)
            if done:
                lat.step(1)  # the first record of a chunk is the state one step after the last one
            a = lat.reduce_series(m, 1)[:, col] / cells / u0
            if stop_below:
                small = np.nonzero(np.abs(a) < stop_below)[0]
                if small.size:
                    out.append(a[:small[0] + 1])
                    break
            out.append(a)
            done += m
        return np.concatenate(out)
    finally:
        lat.close()


def hasimoto_permeability(P, a):
    """k = P^3 / (6 pi a K_H), K_H = 1 / (1 - 1.7601 c^(1/3) + c - 1.5593 c^2), c = 4/3 pi a^3 / P^3."""
    c = 4.0 / 3.0 * math.pi * a ** 3 / P ** 3
    kh = 1.0 / (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2)
    return P ** 3 / (6 * math.pi * a * kh)


def _steady_kapp(lat, check=100, rel_tol=1e-6, max_steps=400000):
    """Step until max|du| over `check` steps falls below rel_tol * max|u| (an FP32 state
    cannot reach a fixed absolute residual far below its rounding of u)."""
    st = None
    for _ in range(max_steps // check):
        lat.step(check)
        st = lat.reduce()
        if st["max_du"] < rel_tol * st["max_u"]:
            break
    return st


def permeability_pair(P, radius_ratio, tau=0.8, F=1e-6, storage=HLBM_F32, width=2.0):
    """Resolved and homogenized apparent permeability of one sphere of radius radius_ratio*P
    in a periodic cell of edge P (steady state), and the dilute-array correlation."""
    from . import inputs
    a = radius_ratio * P
    x = np.arange(P) + 0.5 - P / 2
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    solid = (r < a).astype(np.uint8)
    out = {"P": P, "radius_ratio": radius_ratio, "phi": 1.0 - float(solid.mean())}
    lat = Lattice(HLBM_D3Q19, P, P, P, storage, HLBM_TWO_LATTICE)
    try:
        lat.set_relaxation(tau)
        lat.set_force(F, 0.0, 0.0)
        lat.set_solid_mask(solid)
        lat.init_equilibrium()
        st = _steady_kapp(lat)
        out["k_resolved"] = st["k_app"]
        out["steps_resolved"] = st["step"]
        out["residual_resolved"] = st["max_du"] / st["max_u"]
        lat.set_solid_mask(None)
        lat.set_porosity(inputs.regular_sphere_field(P, period=P, radius_ratio=radius_ratio, width=width))
        lat.init_equilibrium()
        st = _steady_kapp(lat)
        out["k_homogenized"] = st["k_app"]
        out["steps_homogenized"] = st["step"]
        out["residual_homogenized"] = st["max_du"] / st["max_u"]
    finally:
        lat.close()
    a_eff = (3 * float(solid.sum()) / (4 * math.pi)) ** (1 / 3)
    out["a_eff"] = a_eff
    out["k_hasimoto"] = hasimoto_permeability(P, a_eff)
    return out

"""Shared helpers for the GPU parity tests (lattice set-up through the C ABI, error norms)."""
import numpy as np

import paper_2310_14746_gb300 as hb

BC_NAMES = {0: hb.HLBM_PERIODIC, 1: hb.HLBM_HALFWAY_BOUNCE_BACK}


def make_lattice(q, shape, storage=hb.HLBM_F32, pattern=hb.HLBM_TWO_LATTICE, tau=0.6,
                 F=(0.0, 0.0, 0.0), bc=(0, 0, 0), varpi=None, f0=None, scale=None):
    """A lattice of shape (nz, ny, nx) built only through the C ABI."""
    nz, ny, nx = shape
    lat = hb.Lattice(q, nx, ny, nz, storage, pattern)
    lat.set_relaxation(tau)
    lat.set_force(*F)
    for a in range(3):
        lat.set_boundary(a, BC_NAMES[bc[a]])
    if scale is not None:
        lat.set_storage_scale(scale)
    if varpi is not None:
        lat.set_porosity(np.ascontiguousarray(varpi, dtype=np.float32))
    if f0 is not None:
        lat.set_populations(np.ascontiguousarray(f0, dtype=np.float64))
    else:
        lat.init_equilibrium()
    return lat


def rel_inf(a, ref):
    """max |a - ref| / max |ref| (velocity error measure: all cells and components)."""
    return float(np.abs(np.asarray(a, np.float64) - ref).max() / max(np.abs(ref).max(), 1e-300))

"""Reduced-precision storage (FP16 / BF16 deviations from the weights, FP32 arithmetic)
against the FP64 oracle on the random periodic sphere matrix of the 384^3 workload,
resampled at 96^3 (same continuous geometry), 2000 steps.

Stated bounds (velocity max-norm relative error; apparent permeability relative error):
FP16 (scale 2^12) <= 1e-2, BF16 <= 5e-2, FP32 <= 1e-5. Mass drift is monitored by the
FP64 reduction. The measured errors are printed for the record."""
import json
import os

import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice, rel_inf

pytestmark = pytest.mark.gpu

SEED = inputs.SEED_BASE + 3


@pytest.fixture(scope="module")
def reference(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()
    field, info = inputs.random_sphere_field(384, SEED, render_n=96)
    tau, F, steps = 0.6, (1e-6, 0.0, 0.0), 2000
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle.run(oracle.equilibrium_state(19, field.shape), field.astype(np.float64), tau, F, (0, 0, 0), steps)
    _, ur = oracle.moments(ref, F, (0, 0, 0))
    st = oracle.stats(ref, tau, F, (0, 0, 0))
    return dict(field=field, info=info, tau=tau, F=F, steps=steps, u=ur, k_app=st["k_app"])


@pytest.mark.parametrize("storage,bound", [(hb.HLBM_F32, 1e-5), (hb.HLBM_F16DEV, 1e-2), (hb.HLBM_BF16DEV, 5e-2)])
@pytest.mark.parametrize("pattern", [hb.HLBM_TWO_LATTICE, hb.HLBM_AA])
def test_reduced_precision_error_96(reference, storage, bound, pattern):
    r = reference
    lat = make_lattice(19, r["field"].shape, storage, pattern, r["tau"], r["F"], (0, 0, 0), varpi=r["field"])
    lat.step(r["steps"])
    st = lat.reduce()
    _, u = lat.moments()
    lat.close()
    eu = rel_inf(u, r["u"])
    ek = abs(st["k_app"] - r["k_app"]) / abs(r["k_app"])
    drift = st["mass"] / np.prod(r["field"].shape) - 1.0
    print(json.dumps({"storage": hb.STORAGE_NAMES[storage], "pattern": pattern, "velocity_rel_err": eu,
                      "k_app_rel_err": ek, "mass_rel_drift": drift, "k_app_ref": r["k_app"],
                      "field": r["info"]}))
    assert eu <= bound
    assert ek <= bound
    assert abs(drift) < 1e-3


@pytest.mark.parametrize("storage,tol1,tol9", [(hb.HLBM_F16DEV, 1e-4, 5e-4), (hb.HLBM_BF16DEV, 6e-4, 3e-3)])
def test_full_size_384_sampled_cells(oracle, storage, tol1, tol9):
    """The reduced-precision workload at full size, in the launch configuration the bench times
    (384^3, the random Boolean sphere matrix, F along x: the paired two-cells-per-thread kernel,
    a direct launch and then one 8-step graph replay), from a random state near equilibrium,
    f_i = w_i (1 + 0.1 U(-1, 1)). 32 sampled cells are compared with the oracle run on their
    dependency cone (radius 10 around the cell, periodic wrap errors reach 1 cell per step).
    Tolerances are the 16-bit storage rounding: deviations |f - w| <= 0.1 w_i are stored with an
    11-bit (FP16, scaled by 2^12: ulp <= 2^-15 = 3.1e-5 for the rest population, at most 3.8e-6
    for the others) or 8-bit (BF16: ulp <= 2^-12 = 2.4e-4, and 3.1e-5) significand. The initial
    state and every step add at most half an ulp per population; through the density sum and the
    equilibrium (omega = 1/0.6) one step's worst case is about 5e-5 (FP16) and 3.7e-4 (BF16), so
    the bounds are 1e-4 / 6e-4 after 1 step and 5e-4 / 3e-3 after 9. A population taken from the
    wrong neighbour or direction differs by about 0.1 w_i >= 2.8e-3 on this state, far above the
    1-step bounds."""
    import torch
    n, rad, q = 384, 10, 19
    tau, F = 0.6, (1e-6, 0.0, 0.0)
    field, _ = inputs.random_sphere_field(n, SEED)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    rng = np.random.default_rng(SEED + 100)
    f0 = rng.random((q, n, n, n))
    f0 *= 0.2
    f0 += 0.9
    f0 *= w[:, None, None, None]
    cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(32)]
    subs = []
    for z, y, x in cells:
        idx = [np.arange(c - rad, c + rad + 1) % n for c in (z, y, x)]
        subs.append((f0[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]].copy(),
                     field[idx[0]][:, idx[1]][:, :, idx[2]].astype(np.float64)))
    lat = make_lattice(19, (n, n, n), storage, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0), varpi=field, f0=f0)
    del f0
    out = torch.empty((q, n, n, n), dtype=torch.float64, device="cuda")
    zi = torch.tensor([c[0] for c in cells], device="cuda")
    yi = torch.tensor([c[1] for c in cells], device="cuda")
    xi = torch.tensor([c[2] for c in cells], device="cuda")
    done = 0
    for steps, tol in ((1, tol1), (9, tol9)):
        lat.step(steps - done)  # 1 direct launch, then one graph replay of 8
        done = steps
        hb.hlbm_get_populations(lat.h, out)
        torch.cuda.synchronize()
        got = out[:, zi, yi, xi].cpu().numpy()
        for k, (sub, svp) in enumerate(subs):
            ref = oracle.run(sub, svp, tau, F, (0, 0, 0), steps)
            np.testing.assert_allclose(got[:, k], ref[:, rad, rad, rad], rtol=0, atol=tol)
    lat.close()
    del out
    torch.cuda.empty_cache()

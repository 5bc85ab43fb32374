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

"""The two-cells-per-thread step kernel of 16-bit storage against the per-cell kernel:
bit-identical states on periodic lattices whose rows end at every position of a
row segment (one pair, a partial warp, one warp plus one pair, several warps with
idle lanes), for each collision form, over runs that use both single launches
and the captured graph; and the FP16 run of it against the FP64 oracle."""
import os

import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


SHAPES = [(19, (3, 5, 2)), (19, (2, 3, 6)), (19, (4, 7, 30)), (19, (3, 5, 34)), (19, (2, 9, 66)),
          (19, (2, 3, 190)), (19, (2, 2, 194)), (19, (1, 3, 384)), (9, (1, 7, 34)), (9, (1, 5, 130))]
FORMS = ["shift_fx", "shift", "drag", "aniso"]


def _run(q, shape, storage, form, variant, steps=11):
    f0 = inputs.random_populations(q, shape, seed=71, amplitude=0.05)
    vp = inputs.random_porosity(shape, seed=72, lo=0.2)
    F = (1e-4, 0.0, 0.0) if form == "shift_fx" else (1e-4, -2e-4, 3e-4 if q == 19 else 0.0)
    lat = make_lattice(q, shape, storage, hb.HLBM_TWO_LATTICE, 0.7, F, (0, 0, 0), varpi=vp)
    lat.set_step_kernel(variant)
    if form == "drag":
        lat.set_homogenization(hb.HLBM_HOMOG_DRAG)
    if form == "aniso":
        lat.set_porosity_tensor(np.stack([inputs.random_porosity(shape, seed=73 + a, lo=0.2)
                                          for a in range(3)]).astype(np.float32))
    lat.set_populations(f0)
    lat.step(steps)
    out = lat.get_populations()
    lat.close()
    return out


@pytest.mark.parametrize("storage", [hb.HLBM_F16DEV, hb.HLBM_BF16DEV])
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("q,shape", SHAPES)
def test_pair_kernel_bit_identical_to_per_cell(q, shape, form, storage):
    a = _run(q, shape, storage, form, hb.HLBM_STEP_AUTO)
    b = _run(q, shape, storage, form, hb.HLBM_STEP_PER_CELL)
    np.testing.assert_array_equal(a, b)


def test_pair_kernel_fp16_against_oracle(oracle):
    """A 96 x 40 x 24 FP16 run of 200 steps (paired kernel) against the FP64 oracle:
    velocity within the FP16 bound stated for the reduced-precision policy (1e-2)."""
    shape = (24, 40, 96)
    vp = inputs.regular_sphere_field((96, 40, 24), period=8, radius_ratio=0.3)  # (nx, ny, nz)
    F = (1e-5, 0.0, 0.0)
    lat = make_lattice(19, shape, hb.HLBM_F16DEV, hb.HLBM_TWO_LATTICE, 0.6, F, (0, 0, 0), varpi=vp)
    lat.step(200)
    _, u = lat.moments()
    lat.close()
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle.run(oracle.equilibrium_state(19, shape), vp.astype(np.float64), 0.6, F, (0, 0, 0), 200)
    _, ur = oracle.moments(ref, F, (0, 0, 0))
    assert rel_inf(u, ur) < 1e-2

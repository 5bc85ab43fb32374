"""GPU parity of the explicit-drag form of the homogenization (hlbm_set_homogenization) with the
oracle's drag collision; the shift form stays the default."""
import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice, rel_inf

pytestmark = pytest.mark.gpu
DRAG = 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


def _lattice(q, shape, storage, pattern, tau, F, bc, vp, f0=None):
    nz, ny, nx = shape
    lat = hb.Lattice(q, nx, ny, nz, storage, pattern)
    lat.set_relaxation(tau)
    lat.set_force(*F)
    for a in range(3):
        lat.set_boundary(a, hb.HLBM_HALFWAY_BOUNCE_BACK if bc[a] else hb.HLBM_PERIODIC)
    lat.set_homogenization(hb.HLBM_HOMOG_DRAG)
    lat.set_porosity(np.ascontiguousarray(vp, np.float32))
    if f0 is None:
        lat.init_equilibrium()
    else:
        lat.set_populations(f0)
    return lat


@pytest.mark.parametrize("pattern", [hb.HLBM_TWO_LATTICE, hb.HLBM_AA])
@pytest.mark.parametrize("q,shape,bc", [(19, (5, 6, 7), (0, 1, 0)), (19, (3, 4, 33), (1, 0, 1)), (9, (1, 7, 5), (0, 1, 0))])
def test_drag_bruteforce_f64(q, shape, bc, pattern, oracle):
    f0 = inputs.random_populations(q, shape, seed=51)
    vp = inputs.random_porosity(shape, seed=52, lo=0.0)
    F, tau = (2e-4, -1e-4, 3e-4 if q == 19 else 0.0), 0.7
    lat = _lattice(q, shape, hb.HLBM_F64, pattern, tau, F, bc, vp, f0)
    lat.step(17)
    ref = oracle.run_mode(f0, vp.astype(np.float64), tau, F, bc, 17, DRAG)
    np.testing.assert_allclose(lat.get_populations(), ref, rtol=0, atol=1e-13)
    rho, u = lat.moments(f64=True)
    rr, ur = oracle.moments_mode(ref, vp.astype(np.float64), tau, F, bc, DRAG)
    np.testing.assert_allclose(u, ur, rtol=0, atol=1e-13)
    lat.close()


def test_drag_fp32_sphere_field(oracle):
    """FP32 drag form on a sphere field: velocity within 1e-5 of the oracle, and the FP64
    diagnostics' apparent permeability uses the drag-form momentum."""
    n, steps, tau, F = 24, 600, 0.6, (1e-6, 0.0, 0.0)
    vp = inputs.regular_sphere_field(n, period=12, radius_ratio=0.3)
    lat = _lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0), vp)
    lat.step(steps)
    st = lat.reduce()
    _, u = lat.moments()
    lat.close()
    ref = oracle.run_mode(oracle.equilibrium_state(19, (n, n, n)), vp.astype(np.float64), tau, F, (0, 0, 0),
                          steps, DRAG)
    rho, ur = oracle.moments_mode(ref, vp.astype(np.float64), tau, F, (0, 0, 0), DRAG)
    assert rel_inf(u, ur) < 1e-5
    nu = (tau - 0.5) / 3
    k_ref = nu * (rho * ur[0]).mean() / F[0]
    assert abs(st["k_app"] - k_ref) / k_ref < 1e-5


def test_drag_and_shift_share_darcy_limit():
    """Uniform porosity: both forms relax to Darcy's u = F K / nu (K = nu tau / (1 - varpi))."""
    shape, tau, varpi = (4, 4, 4), 0.8, 0.8
    F = (1e-6, 0.0, 0.0)
    K = (tau - 0.5) / 3 * tau / (1 - float(np.float32(varpi)))  # the lattice holds varpi in FP32
    vals = []
    for form in (hb.HLBM_HOMOG_SHIFT, hb.HLBM_HOMOG_DRAG):
        lat = make_lattice(19, shape, hb.HLBM_F64, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0),
                           varpi=np.full(shape, varpi, np.float32))
        lat.set_homogenization(form)
        lat.init_equilibrium()
        lat.step(2000)
        vals.append(lat.reduce()["k_app"])
        lat.close()
    np.testing.assert_allclose(vals, [K, K], rtol=1e-9)


def test_adjoint_refuses_drag_form():
    lat = make_lattice(19, (4, 4, 4))
    lat.set_homogenization(hb.HLBM_HOMOG_DRAG)
    with pytest.raises(hb.HlbmError) as e:
        lat.adjoint_flux_grad(2, 1)
    assert e.value.status == hb.HLBM_ERR_STATE
    lat.close()

"""Resolved obstacles on the GPU (hlbm_set_solid_mask): bounce-back on solid cells against the
oracle, exact equivalence of solid rows with half-way bounce-back walls, and observables."""
import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice

pytestmark = pytest.mark.gpu
PATTERNS = [hb.HLBM_TWO_LATTICE, hb.HLBM_AA]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("q,shape,bc", [(19, (6, 7, 8), (0, 0, 0)), (19, (5, 6, 33), (0, 1, 0)), (9, (1, 9, 12), (1, 0, 0))])
def test_masked_bruteforce_f64(q, shape, bc, pattern, oracle):
    rng = np.random.default_rng(81)
    solid = (rng.random(shape) < 0.25).astype(np.uint8)
    f0 = inputs.random_populations(q, shape, seed=82)
    vp = inputs.random_porosity(shape, seed=83, lo=0.3)
    F, tau = (2e-4, -1e-4, 1e-4 if q == 19 else 0.0), 0.7
    lat = make_lattice(q, shape, hb.HLBM_F64, pattern, tau, F, bc, varpi=vp, f0=f0)
    lat.set_solid_mask(solid)
    lat.step(21)
    ref = oracle.run_masked(f0, vp.astype(np.float64), solid, tau, F, bc, 21)
    fluid = solid == 0
    got = lat.get_populations()
    np.testing.assert_allclose(got[:, fluid], ref[:, fluid], rtol=0, atol=1e-13)
    rho, u = lat.moments(f64=True)
    rr, ur = oracle.moments_masked(ref, solid, F, bc)
    np.testing.assert_allclose(u, ur, rtol=0, atol=1e-13)
    np.testing.assert_allclose(rho, rr, rtol=0, atol=1e-13)
    lat.close()


@pytest.mark.parametrize("pattern", PATTERNS)
def test_solid_rows_equal_walls_fp32(pattern):
    """D2Q9 channel: solid mask rows in a periodic domain give bit-identical fluid rows to the
    half-way bounce-back wall channel (FP32)."""
    H, nx, tau, F = 16, 8, 0.8, (1e-5, 0.0, 0.0)
    vp = np.full((1, H, nx), 0.9, np.float32)
    a = make_lattice(9, (1, H, nx), hb.HLBM_F32, pattern, tau, F, (0, 1, 0), varpi=vp)
    a.step(300)
    vp2 = np.full((1, H + 2, nx), 0.9, np.float32)
    solid = np.zeros((1, H + 2, nx), np.uint8)
    solid[:, 0] = solid[:, H + 1] = 1
    b = make_lattice(9, (1, H + 2, nx), hb.HLBM_F32, pattern, tau, F, (0, 0, 0), varpi=vp2)
    b.set_solid_mask(solid)
    b.init_equilibrium()
    b.step(300)
    _, ua = a.moments()
    _, ub = b.moments()
    np.testing.assert_array_equal(ub[:, :, 1:H + 1, :], ua)
    assert (ub[:, :, 0, :] == 0).all()
    a.close()
    b.close()


def test_resolved_permeability_matches_oracle(oracle):
    """Staircase sphere (radius 3, period 16), FP32, 6000 steps: K_app within 1e-5 of the oracle."""
    P, tau, F = 16, 0.8, (1e-6, 0.0, 0.0)
    x = np.arange(P) + 0.5 - P / 2
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    solid = (r < 3.0).astype(np.uint8)
    lat = make_lattice(19, (P, P, P), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0))
    lat.set_solid_mask(solid)
    lat.init_equilibrium()
    lat.step(6000)
    k = lat.reduce()["k_app"]
    lat.close()
    oracle.set_threads(8)
    f = oracle.run_masked(oracle.equilibrium_state(19, (P, P, P)), np.ones((P, P, P)), solid, tau, F, [0, 0, 0], 6000)
    rho, u = oracle.moments_masked(f, solid, F, [0, 0, 0])
    kr = (tau - 0.5) / 3 * (rho * u[0]).mean() / F[0]
    assert abs(k - kr) / kr < 1e-5


def test_mask_rules():
    lat = make_lattice(19, (4, 4, 4))
    lat.set_solid_mask(np.zeros((4, 4, 4), np.uint8))
    with pytest.raises(hb.HlbmError) as e:
        lat.set_boundary(1, hb.HLBM_HALFWAY_BOUNCE_BACK)
    assert e.value.status == hb.HLBM_ERR_STATE
    with pytest.raises(hb.HlbmError):
        lat.adjoint_flux_grad(2, 1)
    lat.set_solid_mask(None)
    lat.set_boundary(1, hb.HLBM_HALFWAY_BOUNCE_BACK)
    lat.close()

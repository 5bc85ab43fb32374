"""GPU parity of the anisotropic (diagonal-tensor) porosity control with the oracle."""
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


def _tensor(shape, seed):
    return np.stack([inputs.random_porosity(shape, seed + a, lo=0.0) for a in range(3)]).astype(np.float32)


@pytest.mark.parametrize("pattern", [hb.HLBM_TWO_LATTICE, hb.HLBM_AA])
@pytest.mark.parametrize("q,shape,bc", [(19, (5, 6, 7), (0, 1, 0)), (19, (3, 4, 33), (1, 0, 1)), (9, (1, 6, 9), (0, 1, 0))])
def test_aniso_bruteforce_f64(q, shape, bc, pattern, oracle):
    f0 = inputs.random_populations(q, shape, seed=61)
    vp3 = _tensor(shape, 62)
    F, tau = (2e-4, -1e-4, 3e-4 if q == 19 else 0.0), 0.7
    lat = make_lattice(q, shape, hb.HLBM_F64, pattern, tau, F, bc, f0=f0)
    lat.set_porosity_tensor(vp3)
    lat.step(15)
    ref = oracle.run_aniso(f0, vp3.astype(np.float64), tau, F, bc, 15)
    np.testing.assert_allclose(lat.get_populations(), ref, rtol=0, atol=1e-13)
    lat.close()


def test_aniso_fp32_and_isotropic_equivalence(oracle):
    """FP32 tensor run within 1e-5 of the oracle; a tensor with equal components gives the
    same velocity as the scalar field to FP32 rounding."""
    n, steps, tau, F = 20, 400, 0.6, (1e-5, 3e-6, -2e-6)
    vp = inputs.regular_sphere_field(n, period=10, radius_ratio=0.3)
    vp3 = np.stack([vp, np.clip(vp * 0.9 + 0.1, 0, 1), vp ** 2]).astype(np.float32)
    lat = make_lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0))
    lat.set_porosity_tensor(vp3)
    lat.init_equilibrium()
    lat.step(steps)
    _, u = lat.moments()
    ref = oracle.run_aniso(oracle.equilibrium_state(19, (n, n, n)), vp3.astype(np.float64), tau, F, (0, 0, 0), steps)
    _, ur = oracle.moments(ref, F, (0, 0, 0))
    assert rel_inf(u, ur) < 1e-5
    lat.set_porosity_tensor(np.stack([vp, vp, vp]))
    lat.init_equilibrium()
    lat.step(steps)
    _, u3 = lat.moments()
    lat.set_porosity(vp)  # back to the scalar field
    lat.init_equilibrium()
    lat.step(steps)
    _, u1 = lat.moments()
    assert rel_inf(u3, u1) < 1e-6
    lat.close()


def test_aniso_rejections():
    lat = make_lattice(19, (4, 4, 4))
    bad = np.full((3, 4, 4, 4), 0.5, np.float32)
    bad[2, 1, 1, 1] = 1.2
    with pytest.raises(hb.HlbmError):
        lat.set_porosity_tensor(bad)
    lat.set_porosity_tensor(np.full((3, 4, 4, 4), 0.5, np.float32))
    with pytest.raises(hb.HlbmError) as e:
        lat.set_homogenization(hb.HLBM_HOMOG_DRAG)
    assert e.value.status == hb.HLBM_ERR_STATE
    with pytest.raises(hb.HlbmError) as e:
        lat.adjoint_flux_grad(2, 1)
    assert e.value.status == hb.HLBM_ERR_STATE
    lat.close()

"""Time-dependent permeability A~(t) (Darcy law with memory, Sec. 2): relaxation of a periodic
cell from a uniform velocity with no force, on the GPU path, against the oracle and against the
closed form at uniform porosity."""
import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from paper_2310_14746_gb300.workloads import memory_kernel
from hlbm_testutil import make_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


@pytest.mark.parametrize("varpi,tau", [(0.9, 0.8), (0.5, 0.6)])
def test_uniform_porosity_closed_form(varpi, tau):
    """A~_n = (1 - lam)^n exactly and sum A~ = tau/(1 - varpi) = K/nu (FP64 storage)."""
    varpi = float(np.float32(varpi))  # the lattice holds varpi in FP32
    lam = (1 - varpi) / tau
    n = int(40 / lam)
    a = memory_kernel(np.full((4, 4, 4), varpi), tau, n, storage=hb.HLBM_F64)
    np.testing.assert_allclose(a, (1 - lam) ** np.arange(n), rtol=1e-9, atol=1e-15)
    assert abs(a.sum() - tau / (1 - varpi)) / (tau / (1 - varpi)) < 1e-12 + (1 - lam) ** n / lam


def test_sphere_cell_matches_oracle_and_steady_permeability(oracle):
    """24^3 cell of one smoothed sphere (r = 0.3 P): the FP32 A~_n agrees with the oracle's to
    1e-5 (relative to A~_0), and sum A~ agrees with the forced steady K_app / nu within 2e-3
    (the oracle gives the identity to 6e-7 on a 12^3 cell; the bound covers FP32 and the
    truncated tail)."""
    n, tau, u0, steps = 24, 0.6, 1e-4, 20000
    vp = inputs.regular_sphere_field(n, period=24, radius_ratio=0.3)
    a = memory_kernel(vp, tau, steps, u0=u0, stop_below=1e-8)
    f = oracle.equilibrium_state(19, (n, n, n), 1.0, (u0, 0.0, 0.0))
    ref = []
    for k in range(0, 200, 20):
        st = oracle.stats(f, tau, (0, 0, 0), (0, 0, 0))
        ref.append(st["mom_x"] / n ** 3 / u0)
        f = oracle.run(f, vp.astype(np.float64), tau, (0, 0, 0), (0, 0, 0), 20)
    np.testing.assert_allclose(a[0:200:20], ref, rtol=0, atol=1e-5)
    nu = (tau - 0.5) / 3
    lat = make_lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, (1e-6, 0, 0), (0, 0, 0), varpi=vp)
    for _ in range(200):
        lat.step(100)
        st = lat.reduce()
        if st["max_du"] < 1e-10:
            break
    lat.close()
    assert abs(a[-1]) < 1e-6 * a[0]
    assert abs(a.sum() - st["k_app"] / nu) / (st["k_app"] / nu) < 2e-3


def test_reduce_series_equals_reduce_loop():
    """The device-side diagnostics series gives the same records as one hlbm_reduce per sample
    (same kernels), apart from the residual, which the series takes against the unchanged
    reference of the last hlbm_reduce call."""
    import torch
    shape = (6, 7, 40)
    vp = inputs.random_porosity(shape, seed=51, lo=0.3)
    f0 = inputs.random_populations(19, shape, seed=52, amplitude=0.05)
    F = (1e-5, 2e-6, 0.0)
    a = make_lattice(19, shape, hb.HLBM_F32, hb.HLBM_AA, 0.7, F, (0, 1, 0), varpi=vp, f0=f0)
    b = make_lattice(19, shape, hb.HLBM_F32, hb.HLBM_AA, 0.7, F, (0, 1, 0), varpi=vp, f0=f0)
    a.reduce()
    b.reduce()
    rec = a.reduce_series(6, 3)
    dev = torch.empty((6, 8), dtype=torch.float64, device="cuda")
    a.reduce_series(6, 3, out=dev)  # device records, asynchronous
    torch.cuda.synchronize()
    loop = []
    for k in range(6):
        if k:
            b.step(3)
        st = b.reduce()
        loop.append([st[key] for key in hb.STAT_KEYS])
    loop = np.array(loop)
    cols = [0, 1, 2, 3, 4, 5, 7]  # all but max_du
    np.testing.assert_array_equal(rec[:, cols], loop[:, cols])
    a2 = make_lattice(19, shape, hb.HLBM_F32, hb.HLBM_AA, 0.7, F, (0, 1, 0), varpi=vp, f0=f0)
    a2.step(30)  # the second series began where the first one ended (15 steps in)
    st = a2.reduce()
    np.testing.assert_array_equal(dev.cpu().numpy()[5, cols], [st[key] for key in hb.STAT_KEYS if key != "max_du"])
    assert a.steps_taken == 30
    for lat in (a, b, a2):
        lat.close()

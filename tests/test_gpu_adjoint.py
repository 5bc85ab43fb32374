"""GPU adjoint (outflow flux gradient w.r.t. varpi) against the FP64 oracle's reverse sweep
and against central finite differences of FP64 forward runs."""
import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


@pytest.mark.parametrize("shape,bc,every", [((5, 6, 7), (0, 1, 0), 4), ((4, 5, 9), (1, 0, 1), 7),
                                            ((3, 4, 33), (0, 0, 0), 45)])
@pytest.mark.parametrize("pattern", [hb.HLBM_TWO_LATTICE, hb.HLBM_AA])
def test_adjoint_fp64_matches_oracle(shape, bc, every, pattern, oracle):
    """FP64 storage: J and dJ/dvarpi agree with the oracle's reverse sweep to round-off,
    from a random state, with walls, for any recomputation segment length."""
    q, nsteps, tau = 19, 23, 0.7
    f0 = inputs.random_populations(q, shape, seed=31, amplitude=0.3)
    vp = inputs.random_porosity(shape, seed=32, lo=0.1)
    F = (3e-4, -1e-4, 2e-4)
    lat = make_lattice(q, shape, hb.HLBM_F64, pattern, tau, F, bc, varpi=vp, f0=f0)
    J, grad = lat.adjoint_flux_grad(nsteps, every)
    Jr, gr = oracle.flux_grad(f0, vp.astype(np.float64), tau, F, bc, nsteps, every=every)
    assert abs(J - Jr) < 1e-12 * max(1.0, abs(Jr))
    np.testing.assert_allclose(grad, gr, rtol=0, atol=1e-6 * np.abs(gr).max())
    # the state advanced by nsteps
    assert lat.steps_taken == nsteps
    np.testing.assert_allclose(lat.get_populations(), oracle.run(f0, vp.astype(np.float64), tau, F, bc, nsteps),
                               rtol=0, atol=1e-13)
    lat.close()


def test_adjoint_fp32_vs_oracle_24(oracle):
    """Config of the adjoint workload at the oracle's size: 24^3, regular spheres (period 12,
    r = 0.3 P), tau = 0.6, F = 1e-6, 2000 steps, checkpoints every 45 steps. FP32 GPU
    gradient within 1e-4 relative (max-norm) of the FP64 oracle gradient."""
    n, nsteps = 24, 2000
    tau, F = 0.6, (1e-6, 0.0, 0.0)
    vp = inputs.regular_sphere_field(n, period=12, radius_ratio=0.3)
    lat = make_lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0), varpi=vp)
    J, grad = lat.adjoint_flux_grad(nsteps, 45)
    import os
    oracle.set_threads(os.cpu_count() or 1)
    Jr, gr = oracle.flux_grad(oracle.equilibrium_state(19, (n, n, n)), vp.astype(np.float64), tau, F, (0, 0, 0),
                              nsteps, every=45)
    assert abs(J - Jr) / abs(Jr) < 1e-5
    err = np.abs(grad - gr).max() / np.abs(gr).max()
    assert err < 1e-4, err
    lat.close()


def test_autograd_function_matches_direct_call():
    import torch
    from paper_2310_14746_gb300.autograd import HBGKFluxGrad
    n = 16
    vp = torch.from_numpy(inputs.regular_sphere_field(n, period=8, radius_ratio=0.3)).cuda()
    cfg = dict(tau=0.6, F=(1e-5, 0.0, 0.0), nsteps=60, ckpt_every=9)
    v = vp.clone().requires_grad_(True)
    J = HBGKFluxGrad.apply(v, cfg)
    (3.0 * J).backward()
    lat = make_lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, 0.6, cfg["F"], (0, 0, 0),
                       varpi=vp.cpu().numpy())
    J2, g2 = lat.adjoint_flux_grad(60, 9)
    assert float(J.item()) == J2
    np.testing.assert_array_equal(v.grad.cpu().numpy(), 3.0 * g2)
    with torch.no_grad():
        J3 = HBGKFluxGrad.apply(vp, cfg)
    assert float(J3.item()) == J2


def _fd_derivative(J_at, v0, h):
    """dJ/dvarpi at v0 from FP64 forward runs: nodes v0 +- h where both stay in [0, 1] (central),
    else v0 + s h and v0 + 2 s h on the side that does (second-order one-sided). The lattice
    holds varpi in FP32, so every stencil takes the spacing of the rounded values: the
    three-point Lagrange derivative through J(v0) and the two nodes, exact for a quadratic."""
    def node(dv):
        return float(np.float32(v0 + dv)) - v0
    if v0 - h >= 0 and v0 + h <= 1:
        d1, d2 = h, -h
    else:
        s = -1.0 if v0 + h > 1 else 1.0
        d1, d2 = s * h, 2 * s * h
    a1, a2 = node(d1), node(d2)
    l0 = -(a1 + a2) / (a1 * a2)
    l1 = -a2 / (a1 * (a1 - a2))
    l2 = -a1 / (a2 * (a2 - a1))
    return l0 * J_at(0.0) + l1 * J_at(d1) + l2 * J_at(d2)


def test_fd_derivative_stencils():
    """The stencils are exact for a quadratic in the rounded coordinate."""
    for v0 in (0.0, 1.0, float(np.float32(0.37)), float(np.float32(0.9993)), float(np.float32(3e-4))):
        def J_at(dv):
            x = float(np.float32(v0 + dv))
            return 2.0 + 3.0 * x - 5.0 * x * x
        assert abs(_fd_derivative(J_at, v0, 1e-3) - (3.0 - 10.0 * v0)) < 1e-9, v0


def test_adjoint_fd_128_fp64_forwards():
    """Adjoint workload at full size: 128^3, regular spheres (period 32, r = 0.3 P),
    tau = 0.6, F = 1e-6, 2000 steps, checkpoint every 45 steps, FP32 gradient. Checked on
    64 random cells against finite differences of FP64-storage forward runs (h = 1e-3, three-point
    stencils on the rounded spacing): within 1e-3 of the largest sampled |gradient| on every
    cell, and within 1e-2 relative on every cell whose |gradient| exceeds 1e-2 of the largest."""
    n, nsteps, h = 128, 2000, 1e-3
    tau, F = 0.6, (1e-6, 0.0, 0.0)
    vp = inputs.regular_sphere_field(n, period=32, radius_ratio=0.3)
    lat = make_lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0), varpi=vp)
    J32, grad = lat.adjoint_flux_grad(nsteps, 45)
    lat.close()
    fwd = make_lattice(19, (n, n, n), hb.HLBM_F64, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0), varpi=vp)
    dummy = np.empty((n, n, n), np.float32)

    def J_of(field):
        fwd.set_porosity(field)
        fwd.init_equilibrium()
        fwd.step(nsteps)
        J, _ = fwd.adjoint_flux_grad(0, 1, n - 1, dummy)
        return J

    J0 = J_of(vp)
    assert abs(J0 - J32) / abs(J0) < 1e-4
    rng = np.random.default_rng(2310147465)
    cells = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(64)]
    fd, ad = [], []
    for c in cells:
        v0 = float(vp[c])

        def J_at(dv):
            if dv == 0.0:
                return J0
            f = vp.copy()
            f[c] = np.float32(v0 + dv)
            return J_of(f)
        fd.append(_fd_derivative(J_at, v0, h))
        ad.append(float(grad[c]))
    fd, ad = np.array(fd), np.array(ad)
    fwd.close()
    scale = np.abs(fd).max()
    assert scale > 0
    big = np.abs(fd) > 1e-2 * scale
    rel = np.abs(fd - ad)[big] / np.abs(fd)[big]
    print("adjoint 128^3: max |fd - ad| / max |fd| = %.3g; per-cell relative (|fd| > 1e-2 max, %d cells) "
          "max %.3g" % (np.abs(fd - ad).max() / scale, int(big.sum()), rel.max()))
    assert np.abs(fd - ad).max() <= 1e-3 * scale, (fd, ad)
    assert rel.max() <= 1e-2, (fd[big], ad[big])


def test_adjoint_scratch_pool_reuse_and_release():
    """The checkpoints live in the handle's scratch pool: a second gradient from the same state
    reuses the cached memory and gives the same bits, hlbm_release_scratch hands the memory back
    to the device (free memory rises by at least the checkpoints' size), and a gradient after
    the release is again the same."""
    import torch
    n, nsteps, every = 32, 200, 20
    vp = inputs.regular_sphere_field(n, period=16, radius_ratio=0.3)
    lat = make_lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, 0.6, (1e-6, 0.0, 0.0), (0, 0, 0),
                       varpi=vp)
    f0 = lat.get_populations()
    J1, g1 = lat.adjoint_flux_grad(nsteps, every)
    lat.set_populations(f0)
    J2, g2 = lat.adjoint_flux_grad(nsteps, every)
    assert J1 == J2
    np.testing.assert_array_equal(g1, g2)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    lat.release_scratch()
    free_after = torch.cuda.mem_get_info()[0]
    ckpt_bytes = ((nsteps - 1) // every + 1 + every) * 19 * 4 * n ** 3  # snapshots + one segment
    assert free_after - free_before >= 0.9 * ckpt_bytes, (free_after - free_before, ckpt_bytes)
    lat.set_populations(f0)
    J3, g3 = lat.adjoint_flux_grad(nsteps, every)
    assert J3 == J1
    np.testing.assert_array_equal(g3, g1)
    lat.close()

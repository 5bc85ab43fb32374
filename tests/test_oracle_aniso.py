"""Pins of the oracle's anisotropic (diagonal-tensor) porosity control: the Maxwellian at
v = (varpi_x u_x, varpi_y u_y, varpi_z u_z), i.e. a per-axis drag nu/K_a (beyond the isotropy
assumption of Sec. 2.5; anisotropic K is listed as future work in the outlook)."""
import numpy as np
import pytest


def test_isotropic_tensor_equals_scalar(oracle):
    rng = np.random.default_rng(31)
    for q in (9, 19):
        for _ in range(10):
            g = (1 + 0.4 * rng.uniform(-1, 1, q)) / q
            vp, tau = rng.uniform(0, 1), rng.uniform(0.51, 2)
            F = rng.uniform(-1e-3, 1e-3, 3)
            if q == 9:
                F[2] = 0
            np.testing.assert_array_equal(oracle.collide_aniso(q, g, [vp, vp, vp], tau, F),
                                          oracle.collide(q, g, vp, tau, F))


def test_aniso_equilibrium_first_moment_and_budget(oracle):
    """tau = 1, F = 0: the output is M(rho, varpi o u), whose first moment is rho varpi o u; and the
    per-collision momentum change is -((1 - varpi_a)/tau) rho u_a + F_a on each axis."""
    rng = np.random.default_rng(32)
    c, _, _ = oracle.velset(19)
    c = c.astype(float)
    for _ in range(20):
        g = (1 + 0.4 * rng.uniform(-1, 1, 19)) / 19
        vp = rng.uniform(0, 1, 3)
        rho, j = g.sum(), c.T @ g
        m = oracle.collide_aniso(19, g, vp, 1.0, [0, 0, 0])
        np.testing.assert_allclose(c.T @ m, vp * j, atol=1e-16)
        tau = rng.uniform(0.51, 2)
        F = rng.uniform(-1e-3, 1e-3, 3)
        out = oracle.collide_aniso(19, g, vp, tau, F)
        u = (j + F / 2) / rho
        np.testing.assert_allclose(c.T @ out - j, -((1 - vp) / tau) * rho * u + F, atol=2e-16)


@pytest.mark.parametrize("tau", [0.6, 0.9])
def test_aniso_uniform_darcy_per_axis(oracle, tau):
    """Uniform tensor: each axis relaxes independently to Darcy's F_a K_a / nu, K_a = nu tau/(1 - varpi_a)."""
    shape = (3, 4, 5)
    vp3 = np.stack([np.full(shape, v) for v in (0.9, 0.6, 0.3)])
    F = np.array([1e-5, 2e-5, -1e-5])
    lam = (1 - np.array([0.9, 0.6, 0.3])) / tau
    f = oracle.run_aniso(oracle.equilibrium_state(19, shape), vp3, tau, F, [0, 0, 0], int(60 / lam.min()))
    _, u = oracle.moments(f, F, [0, 0, 0])
    for a in range(3):
        np.testing.assert_allclose(u[a], F[a] / lam[a], rtol=1e-10)

"""Pins of the oracle's explicit-drag form of the homogenization (Sec. 3.3, eq.
momentumHLBM: the equilibrium shift acts as the drag -nu K^{-1} rho u; with
varpi = 1 - nu tau / K the drag rate is lam = nu/K = (1 - varpi)/tau)."""
import math

import numpy as np
import pytest

SHIFT, DRAG = 0, 1


@pytest.mark.parametrize("q", [9, 19])
def test_drag_collision_momentum_budget(oracle, q):
    """Per collision mass is conserved and the momentum changes by F - lam rho u with u the
    half-force velocity of the total force, (j + F/2) / (rho (1 + lam/2)); the equilibrium is
    at u itself (no varpi scaling)."""
    rng = np.random.default_rng(21)
    c, w, _ = oracle.velset(q)
    c = c.astype(float)
    dim = 2 if q == 9 else 3
    for _ in range(30):
        g = (1.0 + 0.4 * rng.uniform(-1, 1, q)) / q
        varpi, tau = rng.uniform(0, 1), rng.uniform(0.51, 2.0)
        F = np.zeros(3)
        F[:dim] = rng.uniform(-1e-3, 1e-3, dim)
        out = oracle.collide_mode(q, g, varpi, tau, F, DRAG)
        rho, j = g.sum(), c.T @ g
        lam = (1 - varpi) / tau
        u = (j + F / 2) / (rho * (1 + lam / 2))
        assert abs(out.sum() - rho) < 1e-15
        np.testing.assert_allclose(c.T @ out - j, F - lam * rho * u, atol=2e-16)


@pytest.mark.parametrize("q", [9, 19])
def test_drag_equals_shift_in_free_fluid(oracle, q):
    """At varpi = 1 both forms are plain BGK with Guo forcing: identical collisions."""
    rng = np.random.default_rng(22)
    for _ in range(10):
        g = (1.0 + 0.4 * rng.uniform(-1, 1, q)) / q
        F = rng.uniform(-1e-3, 1e-3, 3)
        if q == 9:
            F[2] = 0
        np.testing.assert_array_equal(oracle.collide_mode(q, g, 1.0, 0.7, F, DRAG),
                                      oracle.collide_mode(q, g, 1.0, 0.7, F, SHIFT))


@pytest.mark.parametrize("varpi,tau", [(0.9, 0.8), (0.5, 0.6), (0.0, 0.55), (0.97, 1.3)])
def test_drag_uniform_box_closed_form(oracle, varpi, tau):
    """Uniform periodic box from rest: u_{n+1} = r u_n + F/(1 + lam/2), r = (1 - lam/2)/(1 + lam/2),
    u_0 = (F/2)/(1 + lam/2); the fixed point is Darcy's F/lam = F K / nu, as for the shift form."""
    q, shape = 19, (3, 4, 5)
    F = np.array([1e-4, -5e-5, 2e-5])
    lam = (1 - varpi) / tau
    r = (1 - lam / 2) / (1 + lam / 2)
    f = oracle.equilibrium_state(q, shape)
    vp = np.full(shape, varpi)
    u = (F / 2) / (1 + lam / 2)
    done = 0
    for n in (1, 9, 60):
        f = oracle.run_mode(f, vp, tau, F, [0, 0, 0], n - done, DRAG)
        for _ in range(n - done):
            u = r * u + F / (1 + lam / 2)
        done = n
        rho, uu = oracle.moments_mode(f, vp, tau, F, [0, 0, 0], DRAG)
        np.testing.assert_allclose(rho, 1.0, atol=1e-14)
        for a in range(3):
            np.testing.assert_allclose(uu[a], u[a], rtol=1e-11, atol=1e-18)
    steady = oracle.run_mode(f, vp, tau, F, [0, 0, 0], int(80 / lam), DRAG)
    _, us = oracle.moments_mode(steady, vp, tau, F, [0, 0, 0], DRAG)
    np.testing.assert_allclose(us[0], F[0] / lam, rtol=1e-9)


def test_drag_brinkman_channel(oracle):
    """Config-1 channel (varpi = 0.9, tau = 0.8, F = 1e-6, H = 32) with the drag form: the profile
    approaches the continuous Brinkman solution of eq. targetEBTL within 1.5e-2 relative L2, and
    the channel centre carries Darcy's g/lam."""
    H, tau, varpi, g = 32, 0.8, 0.9, 1e-6
    nu, lam = (tau - 0.5) / 3, (1 - varpi) / tau
    k = math.sqrt(lam / nu)
    shape = (1, H, 4)
    F = np.array([g, 0.0, 0.0])
    vp = np.full(shape, varpi)
    f = oracle.run_mode(oracle.equilibrium_state(9, shape), vp, tau, F, [0, 1, 0], 5000, DRAG)
    _, u = oracle.moments_mode(f, vp, tau, F, [0, 1, 0], DRAG)
    ux = u[0, 0, :, 0]
    y = np.arange(H) + 0.5
    expect = (g / lam) * (1 - np.cosh(k * (y - H / 2)) / np.cosh(k * H / 2))
    assert np.linalg.norm(ux - expect) / np.linalg.norm(expect) < 1.5e-2
    np.testing.assert_allclose(ux[H // 2], g / lam, rtol=1e-6)

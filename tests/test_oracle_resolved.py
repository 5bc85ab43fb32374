"""Pins of the oracle's resolved-obstacle path (bounce-back on solid cells, varpi = 1 in the
fluid): the pore-scale problem whose permeability the homogenized field stands in for
(Thm. thmStatNSECase4, unit-cell problem for A)."""
import math

import numpy as np
import pytest


def test_solid_rows_equal_halfway_walls(oracle):
    """A channel bounded by solid mask rows (periodic domain) is bit-identical, in its fluid
    rows, to the channel with half-way bounce-back domain walls."""
    H, nx, tau, F = 12, 5, 0.7, (1e-5, 0.0, 0.0)
    rng = np.random.default_rng(71)
    f_in = (1 + 0.3 * rng.uniform(-1, 1, (9, 1, H, nx))) / 9
    wall = oracle.run(f_in, np.ones((1, H, nx)), tau, F, [0, 1, 0], 40)
    solid = np.zeros((1, H + 2, nx), np.uint8)
    solid[:, 0, :] = 1
    solid[:, H + 1, :] = 1
    f_m = np.concatenate([np.full((9, 1, 1, nx), 1 / 9), f_in, np.full((9, 1, 1, nx), 1 / 9)], axis=2)
    masked = oracle.run_masked(f_m, np.ones((1, H + 2, nx)), solid, tau, F, [0, 0, 0], 40)
    np.testing.assert_array_equal(masked[:, :, 1:H + 1, :], wall)
    rho, u = oracle.moments_masked(masked, solid, F, [0, 0, 0])
    assert (u[:, :, 0, :] == 0).all() and (rho[:, 0, :] == 1).all()


def test_masked_run_conserves_fluid_mass(oracle):
    q, shape = 19, (6, 7, 8)
    rng = np.random.default_rng(72)
    solid = (rng.random(shape) < 0.2).astype(np.uint8)
    f = (1 + 0.3 * rng.uniform(-1, 1, (q,) + shape)) / q
    out = oracle.run_masked(f, np.ones(shape), solid, 0.8, (1e-4, 0, 0), [0, 0, 0], 30)
    fluid = solid == 0
    assert abs(out[:, fluid].sum() - f[:, fluid].sum()) < 1e-12


def hasimoto_permeability(P, a):
    """Permeability of a simple cubic array of spheres (period P, radius a) from the dilute drag
    expansion F / (6 pi mu a U) = 1 / (1 - 1.7601 c^(1/3) + c - 1.5593 c^2) (Hasimoto; Sangani &
    Acrivos), c = (4/3) pi a^3 / P^3: k = P^3 / (6 pi a K_H)."""
    c = 4.0 / 3.0 * math.pi * a ** 3 / P ** 3
    kh = 1.0 / (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2)
    return P ** 3 / (6 * math.pi * a * kh)


@pytest.mark.parametrize("a", [2.0, 3.0, 4.0])
def test_resolved_sphere_permeability_vs_hasimoto(oracle, a):
    """A staircase sphere (period 16) with bounce-back: the steady apparent permeability is within
    5 % of the dilute-array correlation evaluated at the volume-equivalent radius of the voxel
    sphere (measured: -0.9 %, -3.0 %, -3.3 % for radii 2, 3, 4)."""
    P, tau = 16, 0.8
    x = np.arange(P) + 0.5 - P / 2
    r = np.sqrt(x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    solid = (r < a).astype(np.uint8)
    F = (1e-6, 0.0, 0.0)
    oracle.set_threads(8)
    f = oracle.run_masked(oracle.equilibrium_state(19, (P, P, P)), np.ones((P, P, P)), solid, tau, F,
                          [0, 0, 0], 6000)
    rho, u = oracle.moments_masked(f, solid, F, [0, 0, 0])
    nu = (tau - 0.5) / 3
    k = nu * (rho * u[0]).mean() / F[0]
    a_eff = (3 * solid.sum() / (4 * math.pi)) ** (1 / 3)
    kh = hasimoto_permeability(P, a_eff)
    assert abs(k - kh) / kh < 0.05, (k, kh)

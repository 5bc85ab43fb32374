"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: lattice
isotropy identities, the moments of the homogenized Maxwellian (Sec. 3.2,
eqs. hbgk statistic equilibrium 1-3), the momentum balance of Sec. 3.3
(eq. momentumHLBM), closed forms of the uniform box and of Darcy's law,
the literature Poiseuille profile with half-way bounce-back, the continuous
Brinkman channel solution of eq. targetEBTL, numpy's roll for streaming, and
central finite differences for the adjoint.
"""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# lattice tables
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q,dim", [(9, 2), (19, 3)])
def test_velset_isotropy(oracle, q, dim):
    """Moments of the weights up to fourth order (c_s^2 = 1/3): these fail for any
    wrong weight, missing or duplicated velocity."""
    c, w, opp = oracle.velset(q)
    c = c.astype(float)[:, :dim]
    assert len(set(map(tuple, c))) == q
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(dim) / 3.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    d = np.eye(dim)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
            + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-16)
    np.testing.assert_array_equal(c[opp], -c)


# --------------------------------------------------------------------------
# homogenized Maxwellian and collision (Sec. 3.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q", [9, 19])
def test_homogenized_maxwellian_moments(oracle, q):
    """With tau = 1 and F = 0 the collision output is M_eq(rho, varpi u) itself.
    Its density is rho, its velocity varpi*u and its pressure rho c_s^2 (eqs. hbgk
    statistic equilibrium 1-3); its momentum flux is rho/3 I + rho (varpi u)(varpi u)."""
    rng = np.random.default_rng(1)
    c, w, _ = oracle.velset(q)
    c = c.astype(float)
    dim = 2 if q == 9 else 3
    for _ in range(20):
        g = (1.0 + 0.4 * rng.uniform(-1, 1, q)) / q
        varpi = rng.uniform(0.0, 1.0)
        rho = g.sum()
        u = (c.T @ g) / rho
        m = oracle.collide(q, g, varpi, 1.0, [0.0, 0.0, 0.0])
        v = varpi * u
        assert abs(m.sum() - rho) < 1e-15
        np.testing.assert_allclose(c.T @ m, rho * v, atol=1e-15)
        rel = c - v
        P = np.einsum("i,ia,ib->ab", m, rel, rel)[:dim, :dim]
        assert abs(np.trace(P) / dim - rho / 3.0) < 1e-15
        Pi = np.einsum("i,ia,ib->ab", m, c, c)[:dim, :dim]
        np.testing.assert_allclose(Pi, rho / 3.0 * np.eye(dim) + rho * np.outer(v, v)[:dim, :dim],
                                   atol=1e-15)


@pytest.mark.parametrize("q", [9, 19])
def test_plain_bgk_limit(oracle, q):
    """varpi = 1 is classical BGK (Sec. 3.2): with F = 0 the collision conserves mass and
    momentum and relaxes toward the equilibrium at the cell's own velocity."""
    rng = np.random.default_rng(2)
    c, _, _ = oracle.velset(q)
    c = c.astype(float)
    for _ in range(10):
        g = (1.0 + 0.4 * rng.uniform(-1, 1, q)) / q
        tau = rng.uniform(0.51, 2.0)
        out = oracle.collide(q, g, 1.0, tau, [0.0, 0.0, 0.0])
        assert abs(out.sum() - g.sum()) < 1e-15
        np.testing.assert_allclose(c.T @ out, c.T @ g, atol=1e-15)
        feq = oracle.equilibrium(q, g.sum(), (c.T @ g) / g.sum())
        np.testing.assert_allclose(out, g - (g - feq) / tau, atol=1e-15)


@pytest.mark.parametrize("q", [9, 19])
def test_collision_momentum_budget(oracle, q):
    """Per collision, mass is conserved and the momentum changes by
    -((1 - varpi)/tau) rho u + F: the homogenization term of eq. momentumHLBM
    (-(1/tau)(rho u - varpi rho u) = -nu K^{-1} rho u) plus the body force, with u the
    half-force velocity (j + F/2)/rho."""
    rng = np.random.default_rng(3)
    c, _, _ = oracle.velset(q)
    c = c.astype(float)
    dim = 2 if q == 9 else 3
    for _ in range(30):
        g = (1.0 + 0.4 * rng.uniform(-1, 1, q)) / q
        varpi = rng.uniform(0.0, 1.0)
        tau = rng.uniform(0.51, 2.0)
        F = np.zeros(3)
        F[:dim] = rng.uniform(-1e-3, 1e-3, dim)
        out = oracle.collide(q, g, varpi, tau, F)
        rho = g.sum()
        j = c.T @ g
        u = (j + F / 2) / rho
        assert abs(out.sum() - rho) < 1e-15
        np.testing.assert_allclose(c.T @ out - j, -((1 - varpi) / tau) * rho * u + F, atol=2e-16)


def test_permeability_relation(oracle):
    """eq. d definition varpi = 1 - nu tau / K, and with the diffusive scaling
    tau = 3 nu eps^2 it becomes eq. bgkPorousity varpi_eps = 1 - 3 nu^2 eps^2 / K."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    assert "bgkPorousity" in gold["scaled_porosity_control"]["citation"]
    nu, eps = 0.05, 0.3
    tau = 3 * nu * eps ** 2
    K = np.array([1e-3, 1e-2, 0.1, 1.0, np.inf, -1.0, 0.0, nu * tau, nu * tau / 2])
    v = oracle.porosity_from_permeability(K, nu, tau)
    expect = np.clip(1 - 3 * nu ** 2 * eps ** 2 / np.where(K > 0, K, 1e-300), 0, 1)
    np.testing.assert_allclose(v, expect, atol=1e-15)
    assert v[4] == gold["plain_bgk_limit"]["value"]  # K -> infinity: plain BGK
    assert v[7] == 0.0 and v[8] == 0.0 and v[5] == 0.0 and v[6] == 0.0


# --------------------------------------------------------------------------
# streaming
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q,shape", [(9, (1, 5, 7)), (19, (4, 5, 6))])
def test_periodic_streaming_is_roll(oracle, q, shape):
    """Periodic pull streaming g_i(x) = f_i(x - c_i) equals numpy's roll by +c_i."""
    rng = np.random.default_rng(4)
    c, _, _ = oracle.velset(q)
    f = rng.random((q,) + shape)
    g = oracle.stream(f, [0, 0, 0])
    for i in range(q):
        expect = np.roll(f[i], shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
        np.testing.assert_array_equal(g[i], expect)


def test_bounce_back_streaming(oracle):
    """With walls on y, a population whose source lies beyond the wall comes back
    from the same cell's opposite direction; all others stream as in the periodic case,
    and the total of each cell column's populations is conserved."""
    q = 9
    rng = np.random.default_rng(5)
    c, _, opp = oracle.velset(q)
    f = rng.random((q, 1, 6, 5))
    g = oracle.stream(f, [0, 1, 0])
    ny = 6
    for i in range(q):
        rolled = np.roll(f[i], shift=(c[i, 1], c[i, 0]), axis=(1, 2))
        for y in range(ny):
            src = y - c[i, 1]
            if 0 <= src < ny:
                np.testing.assert_array_equal(g[i, 0, y], rolled[0, y])
            else:
                np.testing.assert_array_equal(g[i, 0, y], f[opp[i], 0, y])
    assert abs(g.sum() - f.sum()) < 1e-12


# --------------------------------------------------------------------------
# closed forms of the scheme
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q,shape,F", [
    (9, (1, 3, 4), (1e-4, -2e-4, 0.0)),
    (19, (3, 4, 5), (1e-4, 5e-5, -2e-4)),
])
@pytest.mark.parametrize("varpi,tau", [(1.0, 0.8), (0.9, 0.6), (0.5, 1.3), (0.0, 0.55)])
def test_uniform_box_closed_form(oracle, q, shape, F, varpi, tau):
    """Uniform periodic box from rest: by the momentum budget the velocity obeys
    u_{n+1} = (1 - lam) u_n + g with lam = (1 - varpi)/tau, u_0 = g/2 (half-force shift),
    so u_n = g/lam + (g/2 - g/lam)(1 - lam)^n, and u_n = g/2 + n g at varpi = 1.
    The density stays 1."""
    F = np.array(F)
    f = oracle.equilibrium_state(q, shape)
    vp = np.full(shape, varpi)
    lam = (1 - varpi) / tau
    n_done = 0
    for n in (1, 7, 50, 200):
        f = oracle.run(f, vp, tau, F, [0, 0, 0], n - n_done)
        n_done = n
        rho, u = oracle.moments(f, F, [0, 0, 0])
        if lam == 0:
            expect = F / 2 + n * F
        else:
            expect = F / lam + (F / 2 - F / lam) * (1 - lam) ** n
        np.testing.assert_allclose(rho, 1.0, atol=1e-14)
        for a in range(3):
            np.testing.assert_allclose(u[a], expect[a], rtol=1e-11, atol=1e-18)


@pytest.mark.parametrize("varpi,tau", [(0.9, 0.8), (0.5, 0.6), (0.99, 1.0)])
def test_darcy_flux_uniform_porosity(oracle, varpi, tau):
    """At uniform porosity the steady velocity is Darcy's u = g K / nu with
    K = nu tau / (1 - varpi) (eq. d definition, Darcy law of Thm. thmStatNSECase4), and the
    apparent permeability nu <rho u_x> / F_x recovers K."""
    q, shape = 19, (2, 3, 4)
    F = np.array([1e-6, 0.0, 0.0])
    nu = (tau - 0.5) / 3
    K = nu * tau / (1 - varpi)
    lam = (1 - varpi) / tau
    n = int(60 / lam) + 10
    f = oracle.run(oracle.equilibrium_state(q, shape), np.full(shape, varpi), tau, F, [0, 0, 0], n)
    st = oracle.stats(f, tau, F, [0, 0, 0])
    _, u = oracle.moments(f, F, [0, 0, 0])
    np.testing.assert_allclose(u[0], F[0] * K / nu, rtol=1e-10)
    assert abs(st["k_app"] - K) / K < 1e-10


def _channel(oracle, varpi, tau, H, nsteps, g=1e-6, nx=1):
    shape = (1, H, nx)
    F = np.array([g, 0.0, 0.0])
    f = oracle.run(oracle.equilibrium_state(9, shape), np.full(shape, varpi), tau, F,
                   [0, 1, 0], nsteps)
    rho, u = oracle.moments(f, F, [0, 1, 0])
    return rho[0, :, 0], u[0, 0, :, 0], u[1, 0, :, 0]


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_poiseuille_halfway_bounce_back(oracle, tau):
    """Plain BGK (varpi = 1) channel with half-way bounce-back walls and Guo forcing:
    the steady profile is the parabola with the known tau-dependent wall slip,
    u(y) = g/(2 nu) y (H - y) + (g/nu)(16 (tau - 1/2)^2 - 3)/24, y = j + 1/2."""
    H, g = 32, 1e-6
    nu = (tau - 0.5) / 3
    T = H * H / (nu * math.pi ** 2)
    rho, ux, uy = _channel(oracle, 1.0, tau, H, int(25 * T), g=g)
    y = np.arange(H) + 0.5
    expect = g / (2 * nu) * y * (H - y) + (g / nu) * (16 * (tau - 0.5) ** 2 - 3) / 24
    np.testing.assert_allclose(ux, expect, rtol=1e-7)
    np.testing.assert_allclose(uy, 0.0, atol=1e-10 * ux.max())
    np.testing.assert_allclose(rho, 1.0, atol=1e-12)


def test_brinkman_channel_config1(oracle):
    """D2Q9 channel 64x32, varpi = 0.9, tau = 0.8, F = 1e-6, x periodic, walls in y:
    the profile approaches the continuous Brinkman solution of eq. targetEBTL
    u = (g/lam)[1 - cosh(k (y - H/2))/cosh(k H/2)], k = sqrt(lam/nu), lam = (1-varpi)/tau.
    The lattice resolves the wall layer with about one cell (k ~ 1.1), so the stated
    tolerance is 1.5e-2 in relative L2. Far from the walls it is Darcy's g/lam."""
    H, tau, varpi, g = 32, 0.8, 0.9, 1e-6
    nu = (tau - 0.5) / 3
    lam = (1 - varpi) / tau
    k = math.sqrt(lam / nu)
    _, ux, _ = _channel(oracle, varpi, tau, H, 5000, g=g, nx=64 // 16)
    y = np.arange(H) + 0.5
    expect = (g / lam) * (1 - np.cosh(k * (y - H / 2)) / np.cosh(k * H / 2))
    rel = np.linalg.norm(ux - expect) / np.linalg.norm(expect)
    assert rel < 1.5e-2
    np.testing.assert_allclose(ux[H // 2], g / lam, rtol=1e-6)


@pytest.mark.parametrize("tau,varpi", [(0.8, 0.9), (0.6, 0.9), (0.8, 0.5), (1.4, 0.8),
                                       (0.55, 0.99)])
def test_brinkman_discrete_balance(oracle, tau, varpi):
    """Interior nodes of the steady channel satisfy a three-point Brinkman balance
    nu_eff (u_{j+1} - 2 u_j + u_{j-1}) - lam u_j + g = 0 with
    nu_eff = varpi nu - (1 - varpi)(1 - tau): a property of this discretization (it
    reduces to the exact central-difference Poiseuille balance at varpi = 1)."""
    H, g = 24, 1e-6
    nu = (tau - 0.5) / 3
    lam = (1 - varpi) / tau
    nu_eff = varpi * nu - (1 - varpi) * (1 - tau)
    T = min(H * H / (max(nu, 1e-3) * math.pi ** 2), 1 / lam)
    _, ux, _ = _channel(oracle, varpi, tau, H, int(40 * T) + 2000, g=g)
    res = nu_eff * (ux[2:] - 2 * ux[1:-1] + ux[:-2]) - lam * ux[1:-1] + g
    assert np.max(np.abs(res)) < 1e-9 * g


# --------------------------------------------------------------------------
# diagnostics
# --------------------------------------------------------------------------

def test_stats_definitions(oracle):
    """Mass, momentum, plane flux, permeability and residual against numpy sums of the
    oracle's own moments (the reduction bookkeeping, not the physics)."""
    q, shape = 19, (3, 4, 5)
    rng = np.random.default_rng(6)
    from paper_2310_14746_gb300 import inputs
    f = inputs.random_populations(q, shape, 7, amplitude=0.2)
    F = np.array([2e-5, -1e-5, 3e-6])
    tau = 0.7
    rho, u = oracle.moments(f, F, [0, 0, 1])
    up = rng.normal(size=u.shape) * 1e-3
    st = oracle.stats(f, tau, F, [0, 0, 1], u_prev=up)
    assert abs(st["mass"] - rho.sum()) < 1e-12
    assert abs(st["mom_x"] - (rho * u[0]).sum()) < 1e-12
    assert abs(st["mom_z"] - (rho * u[2]).sum()) < 1e-12
    assert abs(st["plane_flux"] - (rho[:, :, -1] * u[0, :, :, -1]).sum()) < 1e-13
    nu = (tau - 0.5) / 3
    assert abs(st["k_app"] - nu * (rho * u[0]).mean() / F[0]) < 1e-12
    assert st["max_du"] == np.abs(u - up).max()
    assert st["max_u"] == np.abs(u).max()


def test_mass_conservation_with_walls(oracle):
    """Streaming with bounce-back and the collision both conserve mass exactly."""
    from paper_2310_14746_gb300 import inputs
    q, shape = 19, (4, 5, 6)
    f = inputs.random_populations(q, shape, 8)
    vp = inputs.random_porosity(shape, 9).astype(np.float64)
    F = np.array([1e-4, 2e-4, -1e-4])
    m0 = f.sum()
    f2 = oracle.run(f, vp, 0.7, F, [1, 0, 1], 25)
    assert abs(f2.sum() - m0) < 1e-12


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q,shape,bc,nsteps", [
    (19, (3, 4, 5), [0, 0, 0], 12),
    (19, (4, 3, 5), [0, 1, 1], 10),
    (9, (1, 6, 5), [0, 1, 0], 20),
])
def test_adjoint_matches_central_differences(oracle, q, shape, bc, nsteps):
    """dJ/dvarpi from the reverse sweep (with recomputation, every=4) equals FP64 central
    finite differences of the forward oracle on every cell (h = 1e-5; the FD rounding
    noise, about 1e-16 |J| / h, and its O(h^2) truncation stay below the 1e-6 bound)."""
    from paper_2310_14746_gb300 import inputs
    f0 = inputs.random_populations(q, shape, 10, amplitude=0.3)
    vp = inputs.random_porosity(shape, 11, 0.3, 1.0).astype(np.float64)
    F = np.array([3e-4, -1e-4, 2e-4 if q == 19 else 0.0])
    tau = 0.7
    J, grad = oracle.flux_grad(f0, vp, tau, F, bc, nsteps, every=4)
    fN = oracle.run(f0, vp, tau, F, bc, nsteps)
    assert abs(J - oracle.flux(fN, F, bc)) < 1e-14
    h = 1e-5
    fd = np.zeros(shape)
    for idx in np.ndindex(*shape):
        vp_p = vp.copy()
        vp_p[idx] += h
        vp_m = vp.copy()
        vp_m[idx] -= h
        Jp = oracle.flux(oracle.run(f0, vp_p, tau, F, bc, nsteps), F, bc)
        Jm = oracle.flux(oracle.run(f0, vp_m, tau, F, bc, nsteps), F, bc)
        fd[idx] = (Jp - Jm) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    np.testing.assert_allclose(grad, fd, atol=1e-6 * scale)


def test_adjoint_segment_length_irrelevant(oracle):
    """The recomputation schedule does not change the gradient."""
    from paper_2310_14746_gb300 import inputs
    q, shape = 19, (3, 3, 4)
    f0 = inputs.random_populations(q, shape, 12, amplitude=0.3)
    vp = inputs.random_porosity(shape, 13).astype(np.float64)
    F = np.array([1e-4, 0, 0])
    J1, g1 = oracle.flux_grad(f0, vp, 0.6, F, [0, 0, 0], 17, every=1)
    J2, g2 = oracle.flux_grad(f0, vp, 0.6, F, [0, 0, 0], 17, every=5)
    J3, g3 = oracle.flux_grad(f0, vp, 0.6, F, [0, 0, 0], 17, every=45)
    assert J1 == J2 == J3
    np.testing.assert_allclose(g1, g2, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(g1, g3, rtol=1e-12, atol=1e-18)


# --------------------------------------------------------------------------
# geometry inputs (the paper's printed porosity value)
# --------------------------------------------------------------------------

def test_minimum_porosity_golden():
    """Prop. porosity: one sphere of diameter equal to the cell edge leaves phi = 1 - pi/6,
    printed as 0.4764."""
    from paper_2310_14746_gb300 import inputs
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))
    item = gold["min_porosity_one_sphere_per_cell"]
    phi = inputs.sphere_matrix_porosity(0.5)
    assert round(phi, item["digits"]) == item["value"]
    # a sharp rendering of that sphere (width -> 0) has nearly that void fraction
    field = inputs.regular_sphere_field(64, period=64.0, radius_ratio=0.5, width=1e-9)
    assert abs(field.mean() - phi) < 2e-3

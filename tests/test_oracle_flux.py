"""Pins of the adjoint objective J, the outflow flux of the oracle.

J is the sum over the plane x = nx - 1 of rho*u_x of the streamed state, with rho and
rho*u the moments of Def. moments (Sec. 3.1) and u the half-force velocity, so that
rho*u_x = sum_i c_ix g_i + F_x/2. Each pin ties ``oracle.flux`` to something other than
itself:

  - a hand-derived closed form on an equilibrium state that varies along x, where the
    pull from the neighbouring planes is known exactly (distinguishes the plane, the
    density factor and the half-force term);
  - the uniform periodic box from rest, J = ny nz u_n with the closed-form recursion of the
    momentum budget (eq. momentumHLBM);
  - the steady plain-BGK channel, J = the sum of the analytic Poiseuille profile with the
    half-way bounce-back slip (the Darcy law of Thm. thmStatNSECase4 at varpi = 1 reduces
    to this Stokes flow);
  - the plane-flux diagnostic on random states with walls and a three-component force
    (that diagnostic is pinned to numpy sums of the moments).

The last test plants mistakes in a private copy of the oracle's C source (wrong plane,
dropped half force, velocity instead of momentum, wrong component) and checks that each
mutant fails at least one pin.
"""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_SRC = os.path.join(ROOT, "oracle", "hbgk_oracle.c")


# --------------------------------------------------------------------------
# the pins, written against any flux function flux_fn(f, F, bc) -> J
# --------------------------------------------------------------------------

def _pin_equilibrium_state(oracle, flux_fn, q):
    """A state of equilibria f_i = w_i rho (1 + 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u.u) whose
    rho(x) and u = (u(x), 0, 0) vary along x only, fully periodic. Summing the weights of
    the directions with c_x = +1 (1/6 for D2Q9 and D3Q19) gives, per cell of the plane
    x = nx - 1, sum_i c_ix g_i = rho_a/6 (1 + 3 u_a + 3 u_a^2) - rho_b/6 (1 - 3 u_b + 3 u_b^2)
    with a = nx - 2 (the source of c_x = +1) and b = 0 (the wrapped source of c_x = -1),
    and rho u_x adds F_x/2."""
    nx, ny, nz = 7, 3, (1 if q == 9 else 2)
    x = np.arange(nx)
    rho_x = 1.0 + 0.2 * np.cos(2 * np.pi * x / nx + 0.3)
    u_x = 0.05 * np.sin(2 * np.pi * x / nx + 1.1)
    c, w, _ = oracle.velset(q)
    cu = c[:, 0:1].astype(float) * u_x[None, :]                      # [q][x]
    feq = w[:, None] * rho_x[None, :] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * u_x[None, :] ** 2)
    f = np.broadcast_to(feq[:, None, None, :], (q, nz, ny, nx)).copy()
    F = np.array([3e-4, -2e-4, 1e-4 if q == 19 else 0.0])
    a, b = nx - 2, 0
    per_cell = (rho_x[a] / 6 * (1 + 3 * u_x[a] + 3 * u_x[a] ** 2)
                - rho_x[b] / 6 * (1 - 3 * u_x[b] + 3 * u_x[b] ** 2) + F[0] / 2)
    expect = ny * nz * per_cell
    J = flux_fn(f, F, [0, 0, 0])
    assert abs(J - expect) <= 1e-14 * ny * nz, (J, expect)


def _pin_uniform_box(oracle, flux_fn):
    """Uniform periodic box from rest (rho = 1): u_n = g/lam + (g/2 - g/lam)(1 - lam)^n with
    lam = (1 - varpi)/tau, so J = ny nz u_n."""
    q, shape = 19, (3, 4, 5)
    nz, ny, nx = shape
    varpi, tau = 0.9, 0.6
    F = np.array([2e-5, -1e-5, 4e-6])
    lam = (1 - varpi) / tau
    f = oracle.equilibrium_state(q, shape)
    done = 0
    for n in (0, 1, 13, 80):
        f = oracle.run(f, np.full(shape, varpi), tau, F, [0, 0, 0], n - done)
        done = n
        u_n = F[0] / lam + (F[0] / 2 - F[0] / lam) * (1 - lam) ** n
        J = flux_fn(f, F, [0, 0, 0])
        assert abs(J - ny * nz * u_n) <= 1e-11 * ny * nz * abs(u_n), (n, J, ny * nz * u_n)


def _pin_poiseuille(oracle, flux_fn, tau=0.8):
    """Plain BGK (varpi = 1) D2Q9 channel, x periodic, half-way bounce-back walls in y,
    Guo forcing, run to steady state: J = sum_j u(y_j) with
    u(y) = g/(2 nu) y (H - y) + (g/nu)(16 (tau - 1/2)^2 - 3)/24, y_j = j + 1/2."""
    H, nx, g = 32, 3, 1e-6
    nu = (tau - 0.5) / 3
    T = H * H / (nu * math.pi ** 2)
    shape = (1, H, nx)
    F = np.array([g, 0.0, 0.0])
    f = oracle.run(oracle.equilibrium_state(9, shape), np.ones(shape), tau, F, [0, 1, 0], int(25 * T))
    y = np.arange(H) + 0.5
    expect = float(np.sum(g / (2 * nu) * y * (H - y) + (g / nu) * (16 * (tau - 0.5) ** 2 - 3) / 24))
    J = flux_fn(f, F, [0, 1, 0])
    assert abs(J - expect) <= 1e-7 * expect, (J, expect)


def _pin_plane_flux_random(oracle, flux_fn):
    """Random states (density far from 1) with walls on two axes and a three-component
    force: J equals the plane-flux diagnostic, and numpy's sum over the plane x = nx - 1 of
    the product of the moments."""
    from paper_2310_14746_gb300 import inputs
    for q, shape, bc, seed in ((19, (4, 5, 6), [0, 1, 1], 31), (19, (3, 4, 7), [1, 0, 1], 32),
                               (9, (1, 6, 5), [0, 1, 0], 33)):
        f = inputs.random_populations(q, shape, seed, amplitude=0.4)
        F = np.array([3e-3, -2e-3, 1e-3 if q == 19 else 0.0])
        J = flux_fn(f, F, bc)
        st = oracle.stats(f, 0.7, F, bc)
        rho, u = oracle.moments(f, F, bc)
        direct = float((rho[:, :, -1] * u[0, :, :, -1]).sum())
        assert abs(J - st["plane_flux"]) <= 1e-13, (J, st["plane_flux"])
        assert abs(J - direct) <= 1e-13, (J, direct)


# --------------------------------------------------------------------------
# the pins applied to the oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("q", [9, 19])
def test_flux_equilibrium_state_closed_form(oracle, q):
    _pin_equilibrium_state(oracle, oracle.flux, q)


def test_flux_uniform_box_closed_form(oracle):
    _pin_uniform_box(oracle, oracle.flux)


def test_flux_poiseuille_channel(oracle):
    _pin_poiseuille(oracle, oracle.flux)


def test_flux_equals_plane_flux_diagnostic(oracle):
    _pin_plane_flux_random(oracle, oracle.flux)


def test_flux_grad_objective_is_flux(oracle):
    """The objective the reverse sweep reports is the pinned J of its final state."""
    from paper_2310_14746_gb300 import inputs
    q, shape, bc = 19, (3, 4, 5), [0, 1, 0]
    f0 = inputs.random_populations(q, shape, 34, amplitude=0.2)
    vp = inputs.random_porosity(shape, 35, 0.2, 1.0).astype(np.float64)
    F = np.array([1e-4, 0.0, 0.0])
    J, _ = oracle.flux_grad(f0, vp, 0.7, F, bc, 9, every=4)
    assert J == oracle.flux(oracle.run(f0, vp, 0.7, F, bc, 9), F, bc)


# --------------------------------------------------------------------------
# planted mistakes: every mutant of oracle_flux fails at least one pin
# --------------------------------------------------------------------------

MUTANTS = {
    "plane x = 0": ("nx - 1, y, z, g)", "0, y, z, g)"),
    "plane x = nx - 2": ("nx - 1, y, z, g)", "nx - 2, y, z, g)"),
    "half force dropped": ("or_moments_cell(&vs, g, F, &r, uu);",
                           "{ const double F0[3] = {0.0, 0.0, 0.0}; or_moments_cell(&vs, g, F0, &r, uu); }"),
    "velocity instead of momentum": ("*J += r * uu[0];", "*J += uu[0];"),
    "wrong component": ("*J += r * uu[0];", "*J += r * uu[1];"),
}


def _mutant_flux(tmp_path, name, old, new):
    """Build a private copy of the oracle with one substitution inside oracle_flux and return
    a flux function bound to it."""
    src = open(ORACLE_SRC).read()
    m = re.search(r"\nint oracle_flux\(.*?\n}\n", src, re.S)
    assert m, "oracle_flux not found"
    body = m.group(0)
    assert body.count(old) == 1, (name, old)
    mutated = src[:m.start()] + body.replace(old, new) + src[m.end():]
    tag = re.sub(r"[^a-z0-9]+", "_", name)
    c_path = tmp_path / ("mutant_%s.c" % tag)
    so_path = tmp_path / ("mutant_%s.so" % tag)
    c_path.write_text(mutated)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c99", "-o", str(so_path), str(c_path), "-lm"],
                   check=True)
    lib = ctypes.CDLL(str(so_path))
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.oracle_flux.argtypes = [ctypes.c_int] * 4 + [ip, dp, dp, dp]

    def flux_fn(f, F, bc):
        f = np.ascontiguousarray(f, dtype=np.float64)
        FF = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(3))
        b = np.ascontiguousarray(bc, dtype=np.int32)
        nz, ny, nx = f.shape[1:]
        J = ctypes.c_double(0.0)
        lib.oracle_flux(f.shape[0], nx, ny, nz, b.ctypes.data_as(ip), FF.ctypes.data_as(dp),
                        f.ctypes.data_as(dp), ctypes.byref(J))
        return J.value
    return flux_fn


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_flux_mistake_is_caught(oracle, tmp_path, name):
    old, new = MUTANTS[name]
    flux_fn = _mutant_flux(tmp_path, name, old, new)
    pins = [lambda: _pin_equilibrium_state(oracle, flux_fn, 19),
            lambda: _pin_equilibrium_state(oracle, flux_fn, 9),
            lambda: _pin_uniform_box(oracle, flux_fn),
            lambda: _pin_poiseuille(oracle, flux_fn),
            lambda: _pin_plane_flux_random(oracle, flux_fn)]
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, "mutant '%s' passes every pin of J" % name


def test_unmutated_copy_passes(oracle, tmp_path):
    """The substitution machinery itself leaves a correct oracle correct."""
    flux_fn = _mutant_flux(tmp_path, "identity", "*J += r * uu[0];", "*J += r * uu[0];")
    _pin_equilibrium_state(oracle, flux_fn, 19)
    _pin_uniform_box(oracle, flux_fn)
    _pin_plane_flux_random(oracle, flux_fn)


# --------------------------------------------------------------------------
# the oracle's own rounding drift at the velocity scale of the D2Q9 channel workload
# --------------------------------------------------------------------------

def test_oracle_drift_at_channel_velocity_scale(oracle):
    """The oracle stores raw populations f ~ 0.1, so a velocity of ~1e-5 formed from them
    carries cancellation error. Measured on the uniform box at the channel workload's scale
    (D2Q9 64x32, varpi = 0.9, tau = 0.8, g = 1e-6) against the closed-form recursion over
    5000 steps: about 2.2e-11 relative. The FP64 GPU-vs-oracle bound of the channel parity
    test (1e-9) sits well above this measured floor."""
    q, shape = 9, (1, 32, 64)
    tau, varpi, g = 0.8, 0.9, 1e-6
    F = np.array([g, 0.0, 0.0])
    lam = (1 - varpi) / tau
    f = oracle.run(oracle.equilibrium_state(q, shape), np.full(shape, varpi), tau, F, [0, 0, 0], 5000)
    _, u = oracle.moments(f, F, [0, 0, 0])
    u_n = g / lam + (g / 2 - g / lam) * (1 - lam) ** 5000
    drift = np.abs(u[0] - u_n).max() / u_n
    assert drift < 1e-10, drift

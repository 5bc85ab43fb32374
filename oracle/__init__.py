"""FP64 CPU oracle for the homogenized lattice BGK (HBGK) scheme.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path never
does. It shares no code with the CUDA library: the arithmetic lives in
``hbgk_oracle.c`` (plain loops, double precision) and this module only
marshals numpy arrays into it.

Method (Simonis et al., arXiv:2310.14746, Part I): BGK relaxation toward the
homogenized Maxwellian evaluated at the porosity-scaled velocity varpi*u
(Sec. 3.2, eqs. porousVeloMaxwellian, "d definition", HBGKBE). The lattice
discretization (DdQq, Guo forcing, pull streaming, half-way bounce-back) is the
textbook one; the paper defers it to its Part II.

Array conventions: populations ``f[q][z][y][x]`` (x fastest), porosity
``varpi[z][y][x]``, velocity ``u[3][z][y][x]``; boundary flags ``bc`` per
axis (x, y, z): 0 periodic, 1 half-way bounce-back walls at both ends.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        i, d, L = ctypes.c_int, ctypes.c_double, ctypes.c_long
        lib.oracle_velset.argtypes = [i, _ip, _dp, _ip]
        lib.oracle_equilibrium.argtypes = [i, d, _dp, _dp]
        lib.oracle_collide.argtypes = [i, _dp, d, d, _dp, _dp]
        lib.oracle_stream.argtypes = [i, i, i, i, _ip, _dp, _dp]
        lib.oracle_run.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _dp, _dp, L]
        lib.oracle_moments.argtypes = [i, i, i, i, _ip, _dp, _dp, _dp, _dp]
        lib.oracle_stats.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _dp, _dp]
        lib.oracle_adjoint_step.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _dp, _dp, _dp, _dp]
        lib.oracle_flux_seed.argtypes = [i, i, i, i, _ip, _dp]
        lib.oracle_flux.argtypes = [i, i, i, i, _ip, _dp, _dp, _dp]
        lib.oracle_flux_grad.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _dp, L, i, _dp, _dp]
        lib.oracle_porosity_from_permeability.argtypes = [_dp, d, d, _dp, ctypes.c_int64]
        lib.oracle_collide_mode.argtypes = [i, _dp, d, d, _dp, i, _dp]
        lib.oracle_run_mode.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _dp, _dp, L, i]
        lib.oracle_moments_mode.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _dp, i, _dp, _dp]
        lib.oracle_run_aniso.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _dp, _dp, L]
        lib.oracle_collide_aniso.argtypes = [i, _dp, _dp, d, _dp, _dp]
        _up = ctypes.POINTER(ctypes.c_ubyte)
        lib.oracle_run_masked.argtypes = [i, i, i, i, _ip, d, _dp, _dp, _up, _dp, _dp, L]
        lib.oracle_moments_masked.argtypes = [i, i, i, i, _ip, _dp, _up, _dp, _dp, _dp]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _bc(bc):
    b = np.ascontiguousarray(bc, dtype=np.int32)
    assert b.shape == (3,)
    return b


def _dims(shape):
    """(nz, ny, nx) of a cell array -> (nx, ny, nz)."""
    nz, ny, nx = shape
    return nx, ny, nz


def set_threads(n: int) -> None:
    """Set the OpenMP thread count used by the oracle's step loop."""
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    """OpenMP threads the oracle's step loop uses."""
    return int(_load().oracle_get_threads())


def velset(q):
    """Velocity set (c[q,3] int, w[q], opp[q]) in the documented ordering."""
    lib = _load()
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    opp = np.zeros(q, dtype=np.int32)
    if lib.oracle_velset(q, c.ctypes.data_as(_ip), _p(w), opp.ctypes.data_as(_ip)):
        raise ValueError("q must be 9 or 19")
    return c, w, opp


def equilibrium(q, rho, v):
    """Homogenized Maxwellian populations at density rho and (scaled) velocity v."""
    lib = _load()
    vv = _f64(np.asarray(v, dtype=np.float64).reshape(3))
    out = np.zeros(q)
    lib.oracle_equilibrium(q, float(rho), _p(vv), _p(out))
    return out


def collide(q, g, varpi, tau, F):
    """One cell's HBGK collision of streamed populations g[q]."""
    lib = _load()
    g = _f64(g)
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    out = np.zeros(q)
    lib.oracle_collide(q, _p(g), float(varpi), float(tau), _p(FF), _p(out))
    return out


def stream(f, bc):
    """Pull streaming g = S f of a state f[q][z][y][x]."""
    lib = _load()
    f = _f64(f)
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    b = _bc(bc)
    g = np.empty_like(f)
    lib.oracle_stream(q, nx, ny, nz, b.ctypes.data_as(_ip), _p(f), _p(g))
    return g


def run(f, varpi, tau, F, bc, nsteps):
    """Advance the post-collision state f[q][z][y][x] by nsteps; returns the new state."""
    lib = _load()
    f = _f64(f).copy()
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    vp = _f64(varpi)
    assert vp.shape == f.shape[1:]
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    tmp = np.empty_like(f)
    rc = lib.oracle_run(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(vp), _p(f),
                        _p(tmp), int(nsteps))
    if rc:
        raise ValueError("oracle_run rejected its arguments (q, tau > 1/2)")
    return f


def moments(f, F, bc):
    """Density rho[z][y][x] and velocity u[3][z][y][x] of the streamed state."""
    lib = _load()
    f = _f64(f)
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    rho = np.empty(f.shape[1:])
    u = np.empty((3,) + f.shape[1:])
    lib.oracle_moments(q, nx, ny, nz, b.ctypes.data_as(_ip), _p(FF), _p(f), _p(rho), _p(u))
    return rho, u


STAT_KEYS = ("mass", "mom_x", "mom_y", "mom_z", "plane_flux", "k_app", "max_du", "max_u")


def stats(f, tau, F, bc, u_prev=None):
    """FP64 global diagnostics of a state, as a dict keyed by STAT_KEYS."""
    lib = _load()
    f = _f64(f)
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    out = np.zeros(8)
    up = None if u_prev is None else _f64(u_prev)
    lib.oracle_stats(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(f),
                     None if up is None else _p(up), _p(out))
    return dict(zip(STAT_KEYS, out.tolist()))


def flux(f, F, bc):
    """Outflow flux J = sum over the plane x = nx-1 of rho*u_x."""
    lib = _load()
    f = _f64(f)
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    J = ctypes.c_double(0.0)
    lib.oracle_flux(q, nx, ny, nz, b.ctypes.data_as(_ip), _p(FF), _p(f), ctypes.byref(J))
    return J.value


def flux_seed(q, shape, bc):
    """dJ/df of the final state for the outflow flux J."""
    lib = _load()
    nx, ny, nz = _dims(shape)
    b = _bc(bc)
    lam = np.zeros((q,) + tuple(shape))
    lib.oracle_flux_seed(q, nx, ny, nz, b.ctypes.data_as(_ip), _p(lam))
    return lam


def adjoint_step(f_n, lam_in, varpi, tau, F, bc, grad):
    """One reverse step; returns dJ/df^n and adds dC/dvarpi^T lam into grad (in place)."""
    lib = _load()
    f_n = _f64(f_n)
    lam_in = _f64(lam_in)
    q = f_n.shape[0]
    nx, ny, nz = _dims(f_n.shape[1:])
    vp = _f64(varpi)
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    assert grad.dtype == np.float64 and grad.flags.c_contiguous
    lam_out = np.empty_like(lam_in)
    lib.oracle_adjoint_step(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(vp),
                            _p(f_n), _p(lam_in), _p(lam_out), _p(grad))
    return lam_out


def flux_grad(f0, varpi, tau, F, bc, nsteps, every=45):
    """(J, dJ/dvarpi) after nsteps from f0, by reverse sweep with recomputation."""
    lib = _load()
    f0 = _f64(f0)
    q = f0.shape[0]
    nx, ny, nz = _dims(f0.shape[1:])
    vp = _f64(varpi)
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    J = ctypes.c_double(0.0)
    grad = np.zeros(f0.shape[1:])
    rc = lib.oracle_flux_grad(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(vp),
                              _p(f0), int(nsteps), int(every), ctypes.byref(J), _p(grad))
    if rc:
        raise RuntimeError("oracle_flux_grad failed (%d)" % rc)
    return J.value, grad


SHIFT, DRAG = 0, 1  # homogenization forms: equilibrium shift (eq. porousVeloMaxwellian), explicit drag


def collide_mode(q, g, varpi, tau, F, mode):
    """One cell's collision in the given homogenization form."""
    lib = _load()
    g = _f64(g)
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    out = np.zeros(q)
    if lib.oracle_collide_mode(q, _p(g), float(varpi), float(tau), _p(FF), int(mode), _p(out)):
        raise ValueError("bad mode or q")
    return out


def run_mode(f, varpi, tau, F, bc, nsteps, mode):
    """oracle.run in the given homogenization form."""
    lib = _load()
    f = _f64(f).copy()
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    vp = _f64(varpi)
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    tmp = np.empty_like(f)
    if lib.oracle_run_mode(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(vp), _p(f), _p(tmp),
                           int(nsteps), int(mode)):
        raise ValueError("oracle_run_mode rejected its arguments")
    return f


def moments_mode(f, varpi, tau, F, bc, mode):
    """(rho, u) of a state as the collision of the given form sees them."""
    lib = _load()
    f = _f64(f)
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    vp = _f64(varpi)
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    rho = np.empty(f.shape[1:])
    u = np.empty((3,) + f.shape[1:])
    lib.oracle_moments_mode(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(vp), _p(f), int(mode),
                            _p(rho), _p(u))
    return rho, u


def collide_aniso(q, g, varpi3, tau, F):
    """One cell's collision with a diagonal porosity tensor (varpi_x, varpi_y, varpi_z)."""
    lib = _load()
    g = _f64(g)
    v3 = _f64(np.asarray(varpi3, dtype=np.float64).reshape(3))
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    out = np.zeros(q)
    lib.oracle_collide_aniso(q, _p(g), _p(v3), float(tau), _p(FF), _p(out))
    return out


def run_aniso(f, varpi3, tau, F, bc, nsteps):
    """oracle.run with a per-cell diagonal porosity tensor varpi3[3][z][y][x]."""
    lib = _load()
    f = _f64(f).copy()
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    v3 = _f64(varpi3)
    assert v3.shape == (3,) + f.shape[1:]
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    tmp = np.empty_like(f)
    if lib.oracle_run_aniso(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(v3), _p(f), _p(tmp),
                            int(nsteps)):
        raise ValueError("oracle_run_aniso rejected its arguments")
    return f


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def run_masked(f, varpi, solid, tau, F, bc, nsteps):
    """oracle.run with resolved solid cells (bounce-back on their surfaces)."""
    lib = _load()
    f = _f64(f).copy()
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    vp = _f64(varpi)
    so = _u8(solid)
    assert so.shape == f.shape[1:]
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    tmp = np.empty_like(f)
    if lib.oracle_run_masked(q, nx, ny, nz, b.ctypes.data_as(_ip), float(tau), _p(FF), _p(vp),
                             so.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _p(f), _p(tmp), int(nsteps)):
        raise ValueError("oracle_run_masked rejected its arguments")
    return f


def moments_masked(f, solid, F, bc):
    """(rho, u) with solid cells reported as rho = 1, u = 0."""
    lib = _load()
    f = _f64(f)
    q = f.shape[0]
    nx, ny, nz = _dims(f.shape[1:])
    so = _u8(solid)
    FF = _f64(np.asarray(F, dtype=np.float64).reshape(3))
    b = _bc(bc)
    rho = np.empty(f.shape[1:])
    u = np.empty((3,) + f.shape[1:])
    lib.oracle_moments_masked(q, nx, ny, nz, b.ctypes.data_as(_ip), _p(FF),
                              so.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), _p(f), _p(rho), _p(u))
    return rho, u


def equilibrium_state(q, shape, rho0=1.0, u0=(0.0, 0.0, 0.0)):
    """State with every cell at the equilibrium of (rho0, u0) (no porosity scaling)."""
    feq = equilibrium(q, rho0, u0)
    return np.broadcast_to(feq.reshape((q,) + (1,) * len(shape)), (q,) + tuple(shape)).copy()


def porosity_from_permeability(K, nu, tau):
    """varpi = 1 - nu*tau/K, clamped to [0, 1] (eq. "d definition")."""
    lib = _load()
    K = _f64(K)
    out = np.empty_like(K)
    lib.oracle_porosity_from_permeability(_p(K), float(nu), float(tau), _p(out), K.size)
    return out

"""GPU parity of the HBGK stream-collide path against the FP64 CPU oracle.

Every lattice here is driven through the C ABI (libhlbm.so) via the thin binding;
expected values come from the oracle only. Tolerances:
  - FP64 storage: populations within 1e-13 (absolute, populations are O(0.1)),
  - FP32 deviation storage: velocity within 1e-5 relative (max-norm over cells and
    components, divided by max |u|),
  - integer-like bookkeeping (step counters, layouts) exact.
"""
import os
import tempfile

import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice, rel_inf

pytestmark = pytest.mark.gpu

PATTERNS = [hb.HLBM_TWO_LATTICE, hb.HLBM_AA]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()
    torch.cuda.init()


# ---------------------------------------------------------------------------
# brute force on tiny and ragged lattices (FP64 storage)
# ---------------------------------------------------------------------------

CASES = [
    # q, (nz, ny, nx), bc
    (19, (4, 4, 4), (0, 0, 0)),
    (19, (5, 6, 7), (0, 1, 0)),
    (19, (3, 5, 33), (1, 0, 1)),
    (19, (2, 3, 130), (0, 1, 1)),   # two x tiles of 128 and a ragged tail
    (19, (6, 7, 8), (1, 1, 1)),
    (9, (1, 8, 4), (0, 1, 0)),
    (9, (1, 5, 37), (1, 1, 0)),
]


@pytest.mark.parametrize("pattern", PATTERNS)
@pytest.mark.parametrize("q,shape,bc", CASES)
def test_bruteforce_f64(q, shape, bc, pattern, oracle):
    f0 = inputs.random_populations(q, shape, seed=100 + sum(shape))
    vp = inputs.random_porosity(shape, seed=200 + sum(shape), lo=0.0, hi=1.0)
    F = (2e-4, -1e-4, 3e-4 if q == 19 else 0.0)
    tau = 0.7
    lat = make_lattice(q, shape, hb.HLBM_F64, pattern, tau, F, bc, varpi=vp, f0=f0)
    # stored as f - w and read back as (f - w) + w: exact up to one rounding of w's size
    np.testing.assert_allclose(lat.get_populations(), f0, rtol=0, atol=1e-16)
    ref = f0
    done = 0
    for n in (1, 2, 13, 50):
        lat.step(n - done)
        ref = oracle.run(ref, vp.astype(np.float64), tau, F, bc, n - done)
        done = n
        got = lat.get_populations()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
        assert lat.steps_taken == n
    rho, u = lat.moments(f64=True)
    rr, ur = oracle.moments(ref, F, bc)
    np.testing.assert_allclose(rho, rr, rtol=0, atol=1e-13)
    np.testing.assert_allclose(u, ur, rtol=0, atol=1e-13)
    lat.close()


@pytest.mark.parametrize("storage", [hb.HLBM_F64, hb.HLBM_F32])
def test_stats_match_oracle(storage, oracle):
    q, shape, bc = 19, (6, 5, 40), (0, 1, 0)
    f0 = inputs.random_populations(q, shape, seed=5, amplitude=0.1)
    vp = inputs.random_porosity(shape, seed=6, lo=0.5)
    F, tau = (1e-4, 0.0, 2e-5), 0.8
    lat = make_lattice(q, shape, storage, hb.HLBM_TWO_LATTICE, tau, F, bc, varpi=vp, f0=f0)
    lat.step(7)
    ref = oracle.run(f0, vp.astype(np.float64), tau, F, bc, 7)
    s1 = lat.reduce()
    o1 = oracle.stats(ref, tau, F, bc, u_prev=np.zeros((3,) + shape))
    _, u7 = oracle.moments(ref, F, bc)
    lat.step(3)
    ref2 = oracle.run(ref, vp.astype(np.float64), tau, F, bc, 3)
    s2 = lat.reduce()
    o2 = oracle.stats(ref2, tau, F, bc, u_prev=u7)
    tol = 1e-11 if storage == hb.HLBM_F64 else 2e-5
    cells = float(np.prod(shape))
    nu = (tau - 0.5) / 3
    for s, o in ((s1, o1), (s2, o2)):
        scale = {"mass": cells, "k_app": nu * o["max_u"] / F[0], "max_du": o["max_u"],
                 "max_u": o["max_u"]}
        for k in ("mass", "mom_x", "mom_y", "mom_z", "plane_flux", "k_app", "max_du", "max_u"):
            sc = scale.get(k, cells * o["max_u"])
            assert abs(s[k] - o[k]) <= tol * sc, (k, s[k], o[k])
    assert s2["step"] == 10


# ---------------------------------------------------------------------------
# FP32 deviation storage
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pattern", PATTERNS)
def test_fp32_velocity_parity_random_field(pattern, oracle):
    q, shape, bc = 19, (12, 10, 36), (0, 0, 1)
    vp = inputs.random_porosity(shape, seed=7, lo=0.0)
    F, tau = (1e-5, 2e-6, -3e-6), 0.6
    lat = make_lattice(q, shape, hb.HLBM_F32, pattern, tau, F, bc, varpi=vp)
    lat.step(300)
    ref = oracle.run(oracle.equilibrium_state(q, shape), vp.astype(np.float64), tau, F, bc, 300)
    _, u = lat.moments()
    _, ur = oracle.moments(ref, F, bc)
    assert rel_inf(u, ur) < 1e-5


def test_patterns_bitwise_identical_fp32():
    """AA (in place) and two-lattice streaming do the same per-cell arithmetic on the same
    values, so their states agree bit for bit."""
    q, shape, bc = 19, (9, 11, 45), (0, 1, 0)
    vp = inputs.random_porosity(shape, seed=8, lo=0.2)
    f0 = inputs.random_populations(q, shape, seed=9, amplitude=0.2)
    F = (1e-5, 0, 0)
    a = make_lattice(q, shape, hb.HLBM_F32, hb.HLBM_TWO_LATTICE, 0.6, F, bc, varpi=vp, f0=f0)
    b = make_lattice(q, shape, hb.HLBM_F32, hb.HLBM_AA, 0.6, F, bc, varpi=vp, f0=f0)
    for n in (1, 9, 40):
        a.step(n)
        b.step(n)
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())


@pytest.mark.parametrize("storage", [hb.HLBM_F32, hb.HLBM_F16DEV, hb.HLBM_BF16DEV])
@pytest.mark.parametrize("fx_only", [False, True])
@pytest.mark.parametrize("q,shape", [(19, (3, 4, 5)), (19, (4, 5, 45)), (19, (2, 3, 130)), (19, (3, 2, 256)),
                                     (19, (2, 5, 200)), (19, (3, 3, 2)), (19, (4, 3, 64)), (9, (1, 7, 131)),
                                     (9, (1, 3, 64))])
def test_aa_periodic_bitwise(q, shape, storage, fx_only):
    """Fully periodic lattices (the in-place kernels without wall logic; for 16-bit storage and
    an even nx the paired two-cells-per-thread AA kernels, in both equilibrium-shift forms):
    rows narrower than a warp, one and several 128-cell row segments, ragged last segments, a
    row of a single cell pair. The AA state equals the two-lattice state of the per-cell kernel
    bit for bit after odd and even step counts."""
    vp = inputs.random_porosity(shape, seed=18, lo=0.2)
    f0 = inputs.random_populations(q, shape, seed=19, amplitude=0.2)
    F = (1e-5, 0.0, 0.0) if fx_only else (1e-5, 2e-6, -3e-6 if q == 19 else 0.0)
    a = make_lattice(q, shape, storage, hb.HLBM_TWO_LATTICE, 0.6, F, (0, 0, 0), varpi=vp, f0=f0)
    b = make_lattice(q, shape, storage, hb.HLBM_AA, 0.6, F, (0, 0, 0), varpi=vp, f0=f0)
    a.set_step_kernel(hb.HLBM_STEP_PER_CELL)  # the same per-cell arithmetic as the AA kernels
    for n in (1, 1, 8, 3, 17):
        a.step(n)
        b.step(n)
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    a.close()
    b.close()


@pytest.mark.parametrize("storage,tol", [(hb.HLBM_F64, 1e-10), (hb.HLBM_F32, 1e-5)])
def test_config1_brinkman_channel(storage, tol, oracle):
    """D2Q9 channel 64x32, x periodic, half-way bounce-back walls in y, varpi = 0.9,
    F = 1e-6, tau = 0.8, 5000 steps: velocity vs the oracle, and the profile vs the
    continuous Brinkman solution of eq. targetEBTL (1.5e-2 relative L2).
    The FP64 bound is set by the oracle: it keeps raw populations f ~ 0.1, so the ~1e-5
    velocities formed from them carry cancellation error. Measured: the oracle drifts
    2.2e-11 relative from the closed-form uniform-box recursion at this velocity scale over
    5000 steps (test_oracle_flux.py), and the GPU's FP64 deviations differ from the oracle by
    2.1e-11 here; the bound leaves a factor of about 5."""
    import math
    shape, bc = (1, 32, 64), (0, 1, 0)
    tau, varpi, g = 0.8, 0.9, 1e-6
    vp = np.full(shape, varpi, dtype=np.float32)
    F = (g, 0.0, 0.0)
    for pattern in PATTERNS:
        lat = make_lattice(9, shape, storage, pattern, tau, F, bc, varpi=vp)
        lat.step(5000)
        _, u = lat.moments(f64=True)
        ref = oracle.run(oracle.equilibrium_state(9, shape), vp.astype(np.float64), tau, F, bc, 5000)
        _, ur = oracle.moments(ref, F, bc)
        err = rel_inf(u, ur)
        print("config-1 channel, %s, pattern %d: velocity rel error vs oracle %.3g"
              % (hb.STORAGE_NAMES[storage], pattern, err))
        assert err < tol
        H = 32
        nu = (tau - 0.5) / 3
        lam = (1 - varpi) / tau
        k = math.sqrt(lam / nu)
        y = np.arange(H) + 0.5
        brink = (g / lam) * (1 - np.cosh(k * (y - H / 2)) / np.cosh(k * H / 2))
        prof = u[0, 0, :, :].mean(axis=1)
        assert np.linalg.norm(prof - brink) / np.linalg.norm(brink) < 1.5e-2
        lat.close()


# ---------------------------------------------------------------------------
# full-size workload (256^3 D3Q19, FP32, launch configuration of the benchmark)
# ---------------------------------------------------------------------------

def test_config2_full_size_vs_unit_cell(oracle):
    """256^3 periodic box of 8^3 regular spheres (period 32, r = 0.3 P), tau = 0.6,
    F = 1e-6, FP32, 1000 steps through the same calls the benchmark times. From a
    uniform start the solution keeps the 32-cell period, so the oracle's 32^3 unit cell
    run gives the expected velocity of every one of the 16.7M cells."""
    n, P = 256, 32
    tau, F = 0.6, (1e-6, 0.0, 0.0)
    vp = inputs.regular_sphere_field(n, period=P, radius_ratio=0.3)
    lat = make_lattice(19, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0), varpi=vp)
    for _ in range(10):
        lat.step(100)
        st = lat.reduce()
    _, u = lat.moments()
    cell_vp = inputs.regular_sphere_field(P, period=P, radius_ratio=0.3).astype(np.float64)
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle.run(oracle.equilibrium_state(19, (P, P, P)), cell_vp, tau, F, (0, 0, 0), 1000)
    _, ur = oracle.moments(ref, F, (0, 0, 0))
    tiled = np.tile(ur, (1, n // P, n // P, n // P))
    assert rel_inf(u, tiled) < 1e-5
    ost = oracle.stats(ref, tau, F, (0, 0, 0))
    assert abs(st["k_app"] - ost["k_app"]) / abs(ost["k_app"]) < 1e-5
    assert abs(st["mass"] - n ** 3) / n ** 3 < 1e-6
    assert st["step"] == 1000
    lat.close()


def test_full_size_sampled_cells_random_state(oracle):
    """256^3 from a random state, 10 steps (one 8-step graph replay + 2 direct steps):
    32 sampled cells against the oracle run on the radius-10 neighbourhood of each cell
    (its dependency cone; wrap-around errors at the sub-block edge reach only radius 1)."""
    n, steps, rad = 256, 10, 10
    q = 19
    rng = np.random.default_rng(11)
    f0 = inputs.random_populations(q, (n, n, n), seed=12, amplitude=0.3)
    vp = inputs.random_porosity((n, n, n), seed=13, lo=0.0)
    F, tau = (2e-5, -1e-5, 5e-6), 0.6
    lat = make_lattice(q, (n, n, n), hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, (0, 0, 0), varpi=vp, f0=f0)
    lat.step(steps)
    got = lat.get_populations()
    for _ in range(32):
        z, y, x = (int(v) for v in rng.integers(0, n, 3))
        idx = [np.arange(c - rad, c + rad + 1) % n for c in (z, y, x)]
        sub = f0[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]
        svp = vp[idx[0]][:, idx[1]][:, :, idx[2]].astype(np.float64)
        ref = oracle.run(sub, svp, tau, F, (0, 0, 0), steps)
        np.testing.assert_allclose(got[:, z, y, x], ref[:, rad, rad, rad], rtol=0, atol=2e-7)
    lat.close()


# ---------------------------------------------------------------------------
# state I/O, checkpoint, validation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("pattern", PATTERNS)
def test_checkpoint_resume_bitwise(pattern):
    q, shape, bc = 19, (8, 9, 40), (0, 1, 0)
    vp = inputs.random_porosity(shape, seed=14, lo=0.3)
    F = (1e-5, 0, 0)
    a = make_lattice(q, shape, hb.HLBM_F32, pattern, 0.6, F, bc, varpi=vp)
    a.step(17)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        a.save(path)
        a.step(23)
        b = make_lattice(q, shape, hb.HLBM_F32, pattern, 0.9, (0, 0, 0), (0, 0, 0))
        b.load(path)
        assert b.steps_taken == 17
        b.step(23)
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())
        assert b.steps_taken == 40


def test_invalid_inputs_rejected():
    lat = make_lattice(19, (4, 4, 4))
    bad = np.full((4, 4, 4), 0.5, dtype=np.float32)
    bad[1, 2, 3] = 1.5
    with pytest.raises(hb.HlbmError) as e:
        lat.set_porosity(bad)
    assert e.value.status == hb.HLBM_ERR_INVALID_ARG
    bad[1, 2, 3] = np.nan
    with pytest.raises(hb.HlbmError):
        lat.set_porosity(bad)
    import torch
    dbad = torch.full((4, 4, 4), 0.5, device="cuda")
    dbad[0, 0, 0] = -0.1
    with pytest.raises(hb.HlbmError):
        lat.set_porosity(dbad)
    with pytest.raises(hb.HlbmError):
        lat.set_relaxation(0.5)
    with pytest.raises(hb.HlbmError):
        lat.set_relaxation(float("nan"))
    with pytest.raises(hb.HlbmError):
        lat.step(-1)
    lat.step(0)
    assert lat.steps_taken == 0
    lat.close()


@pytest.mark.parametrize("on_device", [False, True])
def test_rejected_porosity_leaves_field_unchanged(on_device):
    """A rejected field (one value out of [0, 1]) must not replace the accepted one: the
    lattice then steps bit for bit like a lattice that only ever saw the accepted field."""
    import torch
    shape = (6, 8, 10)
    good = inputs.random_porosity(shape, 11)
    bad = inputs.random_porosity(shape, 12)
    bad[3, 4, 5] = 1.25
    ref = make_lattice(19, shape)
    ref.set_porosity(good)
    ref.init_equilibrium()
    lat = make_lattice(19, shape)
    lat.set_porosity(good)
    with pytest.raises(hb.HlbmError) as e:
        lat.set_porosity(torch.from_numpy(bad).cuda() if on_device else bad)
    assert e.value.status == hb.HLBM_ERR_INVALID_ARG
    lat.init_equilibrium()
    ref.step(24)
    lat.step(24)
    np.testing.assert_array_equal(lat.get_populations(), ref.get_populations())
    ref.close()
    lat.close()


@pytest.mark.parametrize("storage,tol", [(hb.HLBM_F64, 1e-15), (hb.HLBM_F32, 1e-7), (hb.HLBM_F16DEV, 1e-4),
                                         (hb.HLBM_BF16DEV, 1e-3)])
@pytest.mark.parametrize("pattern", [hb.HLBM_TWO_LATTICE, hb.HLBM_AA])
@pytest.mark.parametrize("walls", [False, True])
def test_uniform_init_state(storage, tol, pattern, walls, oracle):
    """init_equilibrium (the uniform fill kernel, several z planes per thread; a ragged last
    group of planes) stores the equilibrium of (rho0, u0) in every cell and direction: read back,
    it equals the oracle's equilibrium within the storage's rounding. For the 32- and 16-bit
    policies the read-back state, written again with set_populations, steps bit for bit like
    the filled one (same layout handling in both write kernels)."""
    nz, ny, nx = 13, 6, 10
    rho0, u0 = 1.01, (0.02, -0.01, 0.015)
    a = hb.Lattice(19, nx, ny, nz, storage, pattern)
    b = hb.Lattice(19, nx, ny, nz, storage, pattern)
    for lat in (a, b):
        lat.set_relaxation(0.7)
        if walls:
            lat.set_boundary(1, hb.HLBM_HALFWAY_BOUNCE_BACK)
    a.init_equilibrium(rho0, u0)
    fa = a.get_populations()
    ref = oracle.equilibrium_state(19, (nz, ny, nx), rho0, u0)
    np.testing.assert_allclose(fa, ref, rtol=0, atol=tol)
    if storage != hb.HLBM_F64:
        b.set_populations(fa)
        vp = inputs.random_porosity((nz, ny, nx), 5)
        for lat in (a, b):
            lat.set_porosity(vp)
            lat.step(3)
        np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    a.close()
    b.close()


def test_device_buffers_and_streams():
    """Porosity from a CUDA tensor, moments into CUDA tensors, on a side stream."""
    import torch
    q, shape = 19, (6, 7, 8)
    vp = torch.rand(shape, device="cuda", dtype=torch.float32)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        lat = hb.Lattice(q, 8, 7, 6, hb.HLBM_F32, hb.HLBM_TWO_LATTICE)
        lat.set_relaxation(0.7)
        lat.set_force(1e-4, 0, 0)
        lat.set_porosity(vp)
        lat.init_equilibrium()
        lat.step(20)
        rho = torch.empty(shape, device="cuda")
        u = torch.empty((3,) + shape, device="cuda")
        hb.hlbm_moments(lat.h, rho, u)
    s.synchronize()
    rho_h, u_h = lat.moments()
    np.testing.assert_array_equal(rho.cpu().numpy(), rho_h)
    np.testing.assert_array_equal(u.cpu().numpy(), u_h)
    lat.close()

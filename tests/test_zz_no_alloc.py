"""The allocation-free diagnostics entry point (hlbm_reduce_noalloc).

It serves callers that may not allocate device memory at the point where they need the
diagnostics (code inside an allocator or memory-pool callback, a host that hands the
library a fixed arena, a monitoring hook that must not fail for lack of memory): the
caller owns every buffer and the library's scratch is a fixed array in device memory.
Here its results are compared with the allocating hlbm_reduce on the same state, over two
calls in a row (the second one also checks the residual against the velocity stored by
the first), in the default equilibrium-shift form and in the explicit-drag form with a
random porosity field; a call made after warm-up must leave the device's free memory
unchanged; and every argument the call cannot serve is refused before any launch.

The file name sorts last so that pytest collects it after every other test file: if it
fails, a run that stops at the first failure has already run the rest of the suite. The
tests do not depend on that order; they pass alone in a fresh process as well.
"""
import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice

pytestmark = pytest.mark.gpu

KEYS = ("mass", "mom_x", "mom_y", "mom_z", "plane_flux", "k_app", "max_du", "max_u")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()


def _device_state(lat, weights):
    """The lattice's post-collision state as FP32 deviations on the device (test-side copy)."""
    import torch
    f = lat.get_populations()
    dev = (f - weights.reshape(-1, 1, 1, 1)).astype(np.float32)
    return torch.from_numpy(dev).cuda()


@pytest.mark.parametrize("form", [hb.HLBM_HOMOG_SHIFT, hb.HLBM_HOMOG_DRAG])
def test_noalloc_reduce_matches_hlbm_reduce(oracle, form):
    import torch
    q, shape, bc = 19, (10, 12, 40), (0, 1, 0)
    nz, ny, nx = shape
    tau, F = 0.7, (1e-4, 0.0, 2e-5)
    _, w, _ = oracle.velset(q)
    f0 = inputs.random_populations(q, shape, seed=41, amplitude=0.1)
    vp = inputs.random_porosity(shape, seed=42, lo=0.3)
    lat = make_lattice(q, shape, hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, bc, varpi=vp)
    lat.set_homogenization(form)
    lat.set_populations(f0)
    varpi_dev = torch.from_numpy(vp).cuda()
    u_prev = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    bcs = [hb.HLBM_PERIODIC, hb.HLBM_HALFWAY_BOUNCE_BACK, hb.HLBM_PERIODIC]
    for call in range(2):
        if call:
            lat.step(9)
        ref = lat.reduce()
        state = _device_state(lat, w)
        got = hb.hlbm_reduce_noalloc(q, nx, ny, nz, hb.HLBM_F32, bcs, tau, F, 1.0, state, u_prev, form=form,
                                     varpi=varpi_dev if form == hb.HLBM_HOMOG_DRAG else None)
        torch.cuda.synchronize()
        for k in KEYS:
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-15), (form, call, k, got[k], ref[k])
    # the residual reference now holds the current velocity
    rho, u = lat.moments()
    np.testing.assert_allclose(u_prev.cpu().numpy(), u, rtol=1e-6, atol=1e-9)
    lat.close()


def test_noalloc_allocates_no_device_memory():
    """After a first call (which looks up the scratch array's address), further calls leave
    the device's free memory exactly where it was."""
    import torch
    q, shape = 19, (16, 16, 64)
    nz, ny, nx = shape
    state = torch.from_numpy((inputs.random_populations(q, shape, seed=43, amplitude=0.1) - 1.0 / q)
                             .astype(np.float32)).cuda()
    u_prev = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    args = (q, nx, ny, nz, hb.HLBM_F32, [0, 0, 0], 0.6, (1e-5, 0.0, 0.0), 1.0, state, u_prev)
    hb.hlbm_reduce_noalloc(*args)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        hb.hlbm_reduce_noalloc(*args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def _refused(status, *args, **kw):
    with pytest.raises(hb.HlbmError) as e:
        hb.hlbm_reduce_noalloc(*args, **kw)
    assert e.value.status == status, (e.value.status, status)


def test_noalloc_rejects_lattice_beyond_scratch():
    import torch
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    # 384-cell rows use blocks of 128 x 2 cells over 4 z planes: 384 x 4 x 65532 cells need
    # 3 x 2 x 16383 = 98298 partial blocks, more than the 65536 the scratch holds (refused
    # before any launch, within hlbm_create's size limits and the launch grid limits)
    _refused(hb.HLBM_ERR_SCRATCH_LIMIT, 19, 384, 4, 65532, hb.HLBM_F32, [0, 0, 0], 0.6, (0, 0, 0), 1.0,
             small, small)


def test_noalloc_rejects_invalid_arguments():
    """Each refusal happens on the host before any launch (the buffers are never read)."""
    import torch
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    E = hb.HLBM_ERR_INVALID_ARG
    base = dict(velset=19, nx=8, ny=8, nz=8, storage=hb.HLBM_F32, bc=[0, 0, 0], tau=0.6, F=(0, 0, 0),
                storage_scale=1.0)

    def call(**over):
        a = dict(base, **over)
        form = a.pop("form", 0)
        varpi = a.pop("varpi", None)
        _refused(E, a["velset"], a["nx"], a["ny"], a["nz"], a["storage"], a["bc"], a["tau"], a["F"],
                 a["storage_scale"], small, small, form=form, varpi=varpi)

    # hlbm_create's size limits (launch-grid dimensions)
    call(nz=65536)
    call(nx=128, ny=65536, nz=1)
    call(velset=9, nz=2)
    # the storage-scale rule of hlbm_set_storage_scale
    call(storage_scale=2.0)
    call(storage=hb.HLBM_F16DEV, storage_scale=3.0)
    call(storage=hb.HLBM_F16DEV, storage_scale=2.0 ** 21)
    call(storage=hb.HLBM_F16DEV, storage_scale=0.5)
    # the drag form needs the porosity field; unknown forms are refused
    call(form=hb.HLBM_HOMOG_DRAG, varpi=None)
    call(form=7)
    call(tau=0.5)

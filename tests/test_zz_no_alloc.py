"""The allocation-free diagnostics entry point (hlbm_reduce_noalloc).

It serves callers that may not allocate device memory (allocator callbacks, fixed
arenas, monitoring hooks): the caller owns every buffer and the library's scratch is a
fixed array in device memory. Here its results are compared with the allocating
hlbm_reduce on the same state, over two calls in a row (the second one also checks the
residual against the velocity stored by the first), and an oversized lattice must be
refused with HLBM_ERR_SCRATCH_LIMIT. This file is collected last on purpose."""
import numpy as np
import pytest

import paper_2310_14746_gb300 as hb
from paper_2310_14746_gb300 import inputs
from hlbm_testutil import make_lattice

pytestmark = pytest.mark.gpu

KEYS = ("mass", "mom_x", "mom_y", "mom_z", "plane_flux", "k_app", "max_du", "max_u")


def _device_state(lat, weights):
    """The lattice's post-collision state as FP32 deviations on the device (test-side copy)."""
    import torch
    f = lat.get_populations()
    dev = (f - weights.reshape(-1, 1, 1, 1)).astype(np.float32)
    return torch.from_numpy(dev).cuda()


def test_noalloc_reduce_matches_hlbm_reduce(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_14746_gb300 import build
    build.build()
    q, shape, bc = 19, (10, 12, 40), (0, 1, 0)
    nz, ny, nx = shape
    tau, F = 0.7, (1e-4, 0.0, 2e-5)
    _, w, _ = oracle.velset(q)
    f0 = inputs.random_populations(q, shape, seed=41, amplitude=0.1)
    vp = inputs.random_porosity(shape, seed=42, lo=0.3)
    lat = make_lattice(q, shape, hb.HLBM_F32, hb.HLBM_TWO_LATTICE, tau, F, bc, varpi=vp, f0=f0)
    u_prev = torch.zeros((3,) + shape, dtype=torch.float32, device="cuda")
    bcs = [hb.HLBM_PERIODIC, hb.HLBM_HALFWAY_BOUNCE_BACK, hb.HLBM_PERIODIC]
    for call in range(2):
        if call:
            lat.step(9)
        ref = lat.reduce()
        state = _device_state(lat, w)
        got = hb.hlbm_reduce_noalloc(q, nx, ny, nz, hb.HLBM_F32, bcs, tau, F, 1.0, state, u_prev)
        torch.cuda.synchronize()
        for k in KEYS:
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-15), (call, k, got[k], ref[k])
    # the residual reference now holds the current velocity
    rho, u = lat.moments()
    np.testing.assert_allclose(u_prev.cpu().numpy(), u, rtol=1e-6, atol=1e-9)
    lat.close()


def test_noalloc_rejects_lattice_beyond_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    # 32-cell rows use blocks of 32 x 8 cells over 4 z planes: 32 x 8 x 262145 cells need
    # 65537 partial blocks, one more than the scratch holds (refused before any launch)
    with pytest.raises(hb.HlbmError) as e:
        hb.hlbm_reduce_noalloc(19, 32, 8, 4 * 65536 + 1, hb.HLBM_F32, [0, 0, 0], 0.6, (0, 0, 0), 1.0, small, small)
    assert e.value.status == hb.HLBM_ERR_SCRATCH_LIMIT

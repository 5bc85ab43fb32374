"""torch.autograd.Function for the outflow-flux gradient with respect to varpi.

J(varpi) = sum over the plane x = plane_x of rho*u_x after `nsteps` HBGK steps from
rest, and dJ/dvarpi from the library's hand-written adjoint kernels with checkpointed
recomputation (hlbm_adjoint_flux_grad). varpi is the porosity control of eq.
"d definition" (Simonis et al., arXiv:2310.14746, Part I, Sec. 3.2).
"""
from __future__ import annotations

import numpy as np
import torch

from . import (HLBM_D3Q19, HLBM_F32, HLBM_HALFWAY_BOUNCE_BACK, HLBM_PERIODIC, HLBM_TWO_LATTICE, Lattice)


class HBGKFluxGrad(torch.autograd.Function):
    """J = HBGKFluxGrad.apply(varpi, cfg). varpi: float32 CUDA tensor [nz, ny, nx] in [0, 1].
    cfg keys: tau, F (3-tuple), nsteps, ckpt_every (default 45), plane_x (default nx-1),
    bc (3-tuple of 0 periodic / 1 wall), storage (default FP32), velset (default D3Q19).

    When varpi requires a gradient, forward runs the whole adjoint (forward sweep with
    checkpoints, then the reverse sweep) eagerly and keeps dJ/dvarpi; backward only scales it.
    The reverse sweep needs the forward checkpoints, so deferring it to backward would mean a
    second forward run; a forward whose gradient is never used therefore pays the adjoint's
    cost. With no gradient requested, forward runs the forward steps alone."""

    @staticmethod
    def forward(ctx, varpi, cfg):
        if not varpi.is_cuda or varpi.dtype != torch.float32:
            raise TypeError("varpi must be a float32 CUDA tensor")
        v = varpi.detach().contiguous()
        nz, ny, nx = v.shape
        lat = Lattice(cfg.get("velset", HLBM_D3Q19), nx, ny, nz, cfg.get("storage", HLBM_F32),
                      cfg.get("pattern", HLBM_TWO_LATTICE))
        try:
            lat.set_relaxation(cfg["tau"])
            lat.set_force(*cfg["F"])
            for a, b in enumerate(cfg.get("bc", (0, 0, 0))):
                lat.set_boundary(a, HLBM_HALFWAY_BOUNCE_BACK if b else HLBM_PERIODIC)
            lat.set_porosity(v)
            lat.init_equilibrium()
            plane = cfg.get("plane_x", nx - 1)
            if ctx.needs_input_grad[0]:
                grad = torch.empty_like(v)
                J, _ = lat.adjoint_flux_grad(cfg["nsteps"], cfg.get("ckpt_every", 45), plane, grad)
                ctx.save_for_backward(grad)
            else:
                lat.step(cfg["nsteps"])
                J, _ = lat.adjoint_flux_grad(0, 1, plane, np.empty(v.shape, np.float32))
        finally:
            lat.close()
        return torch.tensor(J, dtype=torch.float64, device=varpi.device)

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return (gJ.to(grad.dtype) * grad), None


def flux_and_grad(varpi: torch.Tensor, **cfg):
    """Convenience: (J, dJ/dvarpi) for a float32 CUDA varpi tensor."""
    v = varpi.detach().clone().requires_grad_(True)
    J = HBGKFluxGrad.apply(v, cfg)
    J.backward()
    return float(J.item()), v.grad

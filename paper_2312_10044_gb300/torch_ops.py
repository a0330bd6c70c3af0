"""PyTorch autograd interface to the solvation energy.

``BipbEnergy.apply(q, pos, surface, params)`` returns the electrostatic
solvation energy E (kcal/mol) of the charges ``q`` (e) at ``pos`` (A) inside
a fixed surface, one value per charge configuration.  Its backward pass
gives dE/dq and dE/dpos from one adjoint GMRES solve A^T lam = c per
configuration and one gradient pass on the GPU (the energy of Sec. 2.2.1,
Eq. for E_sol, differentiated at fixed surface):

    dE/dtheta = 1/2 [ (dc/dtheta) . u + lam . (db/dtheta) ],   A u = b,  E = 1/2 c . u

Torch tensors are only the carriers of the inputs and outputs; every step
runs in libbipb.  CUDA tensors go to the library's device entry points
(bipb_charges_set_dev, bipb_energy_dev, bipb_energy_grad_dev) and never pass
through the host; CPU tensors go through the host entry points.  ``q`` is
(B, Nc) or (Nc,), ``pos`` is (Nc, 3) or (B, Nc, 3).
"""
from __future__ import annotations

import numpy as np
import torch

from . import MIXED, PRECOND_NONE, Surface, solve_params


def _set(surface: Surface, q, pos):
    if q.is_cuda:
        surface.set_charges_dev(pos.detach().to(torch.float64), q.detach().to(torch.float64))
    else:
        surface.set_charges(pos.detach().to(torch.float64).numpy(), q.detach().to(torch.float64).numpy())


class BipbEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q, pos, surface: Surface, params):
        squeeze = q.dim() == 1
        _set(surface, q, pos)
        surface.solve(params)
        if q.is_cuda:
            out = surface.energy_dev().to(q.dtype)
        else:
            out = torch.as_tensor(surface.energy(), dtype=q.dtype)
        ctx.surface = surface
        ctx.params = params
        ctx.squeeze = squeeze
        ctx.pos_batched = pos.dim() == 3
        ctx.version = surface_version(surface)
        ctx.save_for_backward(q, pos)
        return out[0] if squeeze else out

    @staticmethod
    def backward(ctx, grad_e):
        q, pos = ctx.saved_tensors
        s = ctx.surface
        if surface_version(s) != ctx.version:  # the handle was used for other charges since forward
            _set(s, q, pos)
            s.solve(ctx.params)
        if q.is_cuda:
            dq, dy = s.energy_grad_dev(ctx.params)
        else:
            dq, dy = (torch.as_tensor(a) for a in s.energy_grad(ctx.params))
        g = grad_e.detach().to(torch.float64).reshape(-1)
        gq = dq * g[:, None]
        gy = dy * g[:, None, None]
        if not ctx.pos_batched:
            gy = gy.sum(dim=0)
        grad_q = (gq[0] if ctx.squeeze else gq).to(q.dtype)
        return grad_q, gy.to(pos.dtype), None, None


def surface_version(surface: Surface):
    """Identity of the charge set last given to the handle (changes on every set_charges)."""
    return getattr(surface, "_charge_version", None)


class SolvationEnergy(torch.nn.Module):
    """E(q, pos) for charges inside a fixed triangulated surface (kcal/mol).

    The surface is uploaded once; each forward sets the charges, solves
    (mixed precision by default, relative residual ``tol``) and returns the
    energy of every configuration.  Backward runs the adjoint solve.
    """

    def __init__(self, centroids, normals, areas, eps_in=1.0, eps_out=80.0, kappa=0.1257, tol=1e-8,
                 precision=MIXED, restart=10, precond=PRECOND_NONE):
        super().__init__()
        self.surface = Surface(np.asarray(centroids), np.asarray(normals), np.asarray(areas))
        self.params = solve_params(eps_in, eps_out, kappa, tol=tol, restart=restart, precision=precision,
                                   precond=precond)

    def forward(self, q, pos):
        return BipbEnergy.apply(q, pos, self.surface, self.params)

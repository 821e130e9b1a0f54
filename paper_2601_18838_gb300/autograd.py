"""torch.autograd.Function around the reciprocal energy.

Forward calls ``kpme_energy_forces`` once: the gather kernel evaluates the
potentials phi_i and, with the derivative B-splines dM_n/du, the adjoint
-dE/dx_i in the same pass.  Backward therefore needs no second contraction:
  dE/dx_i = -F_i,  dE/dq_i = phi_i  (E is quadratic in q and the mesh operator
  is symmetric).
"""
from __future__ import annotations

import torch


class ReciprocalEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, q, plan):
        out = plan.energy_forces(x.detach().contiguous(), q.detach().contiguous(), forces=True, dEdq=True)
        ctx.save_for_backward(out["forces"], out["dEdq"])
        return out["energy"].reshape(())

    @staticmethod
    def backward(ctx, g):
        F, phi = ctx.saved_tensors
        gx = -g * F if ctx.needs_input_grad[0] else None
        gq = g * phi if ctx.needs_input_grad[1] else None
        return gx, gq, None


def reciprocal_energy(x: torch.Tensor, q: torch.Tensor, plan) -> torch.Tensor:
    """Differentiable reciprocal energy E(x, q) on ``plan`` (a ``Plan``)."""
    return ReciprocalEnergy.apply(x, q, plan)

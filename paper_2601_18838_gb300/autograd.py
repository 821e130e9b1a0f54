"""torch.autograd.Functions around the reciprocal energy and potentials.

Energy: forward calls ``kpme_energy_forces`` once: the gather kernel evaluates
the potentials phi_i and, with the derivative B-splines dM_n/du, the adjoint
-dE/dx_i in the same pass.  Backward therefore needs no second contraction:
  dE/dx_i = -F_i,  dE/dq_i = phi_i  (E is quadratic in q and the mesh operator
  is symmetric).

Potentials at targets X of charges q at sources Y (§1.1, X != Y):
  p = k_e (S_X^T H S_Y q - c sum(q)),
with S the B-spline interpolation matrices, H the symmetric SKP mesh operator and
c its m = 0 correction (0 for the SVD form).  For an upstream gradient g on p:
  dL/dq = k_e (S_Y^T H S_X g - c sum(g))           (the adjoint problem),
  dL/dx_i = g_i k_e grad(S^T H S_Y q)(x_i)          (a gather at X with charges g),
  dL/dy_j = q_j k_e grad(S^T H S_X g)(y_j)          (a gather at Y of the adjoint mesh),
all through the library's spread / apply / gather entry points (apply subtracts c sum(Q)
on the mesh, which the gather's partition of unity carries to every particle).
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


class ReciprocalPotential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, q, x, plan):
        y, q, x = y.detach().contiguous(), q.detach().contiguous(), x.detach().contiguous()
        p = plan.potential(y, q, x)
        ctx.plan = plan
        ctx.save_for_backward(y, q, x)
        return p

    @staticmethod
    def backward(ctx, g):
        y, q, x = ctx.saved_tensors
        plan = ctx.plan
        g = g.detach().contiguous()
        gy = gq = gx = None
        if ctx.needs_input_grad[2]:
            Phi = plan.apply(plan.spread(y, q))
            _, F = plan.gather(x, g, Phi, forces=True)        # F_i = -g_i k_e grad(phi)(x_i)
            gx = -F
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            Phi_adj = plan.apply(plan.spread(x, g))
            phi_adj, F_adj = plan.gather(y, q, Phi_adj, forces=ctx.needs_input_grad[0])
            if ctx.needs_input_grad[1]:
                gq = phi_adj      # apply() includes the -c sum correction, carried by the gather
            if ctx.needs_input_grad[0]:
                gy = -F_adj
        return gy, gq, gx, None


def reciprocal_potential(y: torch.Tensor, q: torch.Tensor, x: torch.Tensor, plan) -> torch.Tensor:
    """Differentiable reciprocal potentials at targets x of charges q at sources y on ``plan``."""
    return ReciprocalPotential.apply(y, q, x, plan)

"""torch.autograd.Function for the through-thickness stress field as a function
of the per-element fibre misalignment angles.

forward:  theta (n_elem, FP64, CUDA) -> s33 (n_elem): sets the angles, runs the
          GenEO-PCG solve and the centre stress recovery (gl_set_theta,
          gl_solve, gl_stress).
backward: g = dL/ds33 -> dL/dtheta by one adjoint PCG solve reusing the
          preconditioner and the element contraction (gl_stress_vjp,
          gl_adjoint).
Any objective built from s33 with torch (for example a p-norm over the resin
elements of the corner) then differentiates through it.  All arithmetic of the
solve, the recovery and the adjoint runs in the CUDA library.
"""
from __future__ import annotations

import torch


class StressOfTheta(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, solver, f):
        theta = theta.detach().contiguous()
        solver.set_theta(theta)
        n, ne = solver.n_dof, solver.n_elem
        u = torch.empty(n, dtype=torch.float64, device=theta.device)
        s33 = torch.empty(ne, dtype=torch.float64, device=theta.device)
        t13 = torch.empty(ne, dtype=torch.float64, device=theta.device)
        solver.solve(f, out=u)
        solver.stress(u, s33, t13)
        ctx.solver = solver
        ctx.save_for_backward(u)
        return s33

    @staticmethod
    def backward(ctx, g33):
        (u,) = ctx.saved_tensors
        s = ctx.solver
        dJdu = torch.empty(s.n_dof, dtype=torch.float64, device=u.device)
        explicit = torch.empty(s.n_elem, dtype=torch.float64, device=u.device)
        s.stress_vjp(u, g33.contiguous(), None, dJdu, explicit)
        grad = torch.empty(s.n_elem, dtype=torch.float64, device=u.device)
        s.adjoint(u, dJdu, grad)
        return grad + explicit, None, None


def stress_of_theta(theta, solver, f=None):
    """s33 per element as a differentiable function of theta (see StressOfTheta)."""
    return StressOfTheta.apply(theta, solver, f)


def pnorm(x, mask, p=8):
    """(sum_{mask} x^p)^(1/p), the aggregated through-thickness stress."""
    return (x[mask] ** p).sum() ** (1.0 / p)

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


def element_dofs(nx, ny, e):
    """The 81 global DOFs of element e of a structured nx x ny x nz Q2 mesh
    (node n = ix + NX (iy + NY iz), x fastest; dof = 3 n + component)."""
    NX, NY = 2 * nx + 1, 2 * ny + 1
    ex, ey, ez = e % nx, (e // nx) % ny, e // (nx * ny)
    out = []
    for k in range(3):
        for j in range(3):
            for i in range(3):
                n = (2 * ex + i) + NX * ((2 * ey + j) + NY * (2 * ez + k))
                out.extend((3 * n, 3 * n + 1, 3 * n + 2))
    return out


def theta_central_differences(solver, nx, ny, theta0, elems, mask, p=8, h=1e-6, f=None):
    """Central differences (J(theta0 + h e_k) - J(theta0 - h e_k)) / 2h of the
    p-norm objective J = (sum_mask s33^p)^(1/p) for each element k in `elems`.

    Every perturbed state is reached by an increment from u0 = u(theta0):
        K(theta) du = -(K(theta) - K(theta0)) u0   (du = 0 on Dirichlet DOFs),
    the right-hand side restricted to element k's DOFs (the only element whose
    stiffness changes), u = u0 + du, so the difference carries the increment
    solve's tolerance and not the residual of u0.  The difference of J is
    evaluated without cancelling large terms: the stresses are linear in u,
    s = a + b with a = s33(theta, u0) (bitwise equal to s33(theta0, u0) except
    at element k) and b = s33(theta, du), and with d = s+ - s- formed from the
    small parts,
        S+ - S- = sum d (x^(p-1) + x^(p-2) y + ... + y^(p-1)),  x = s+, y = s-,
        J+ - J- = (S+ - S-) / (J+^(p-1) + ... + J-^(p-1)),      S = J^p.
    Every product, solve and stress runs in the CUDA library (gl_apply_K,
    gl_solve_increment, gl_stress); the solver's angles are restored."""
    dev = theta0.device
    n, ne = solver.n_dof, solver.n_elem
    solver.set_theta(theta0)
    u0 = torch.empty(n, dtype=torch.float64, device=dev)
    solver.solve(f, out=u0)
    y0 = torch.empty_like(u0)
    solver.apply_K(u0, out=y0)
    y = torch.empty_like(u0)
    g = torch.zeros_like(u0)
    du = torch.empty_like(u0)
    t13 = torch.empty(ne, dtype=torch.float64, device=dev)
    out = []
    try:
        for k in elems:
            idx = torch.tensor(element_dofs(nx, ny, int(k)), device=dev)
            parts = []
            for sgn in (1.0, -1.0):
                th = theta0.clone()
                th[int(k)] += sgn * h
                solver.set_theta(th)
                solver.apply_K(u0, out=y)
                g.zero_()
                g[idx] = y0[idx] - y[idx]
                solver.solve_increment(g, out=du)
                a = torch.empty(ne, dtype=torch.float64, device=dev)
                b = torch.empty(ne, dtype=torch.float64, device=dev)
                solver.stress(u0, a, t13)
                solver.stress(du, b, t13)
                parts.append((a[mask], b[mask]))
            (ap, bp), (am, bm) = parts
            d = (ap - am) + (bp - bm)
            x, z = ap + bp, am + bm
            poly = sum(x ** (p - 1 - i) * z ** i for i in range(p))
            dS = (d * poly).sum()
            Jp, Jm = (x ** p).sum() ** (1.0 / p), (z ** p).sum() ** (1.0 / p)
            dJ = dS / sum(Jp ** (p - 1 - i) * Jm ** i for i in range(p))
            out.append(dJ.item() / (2.0 * h))
    finally:
        solver.set_theta(theta0)
    return out

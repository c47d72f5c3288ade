"""Oracle gradient of a stress objective with respect to the misalignment angles.

Test infrastructure only (see the package docstring).  Plain FP64 SciPy with
direct solves (no CG error).

Objective (the corner-unfolding study of Section 3 assesses the
through-thickness stress sigma_r = sigma_33 in the resin interfaces, Eq.
eq-Camanho): J(theta) = (sum_{e in E} s33_e^p)^(1/p), s33_e the element-centre
sigma_rr of the recovered stress.

Adjoint (standard, written out): with K(theta) u = f on the free DOFs,
  dJ/dtheta_e = dJ/dtheta_e|_u - lambda_e^T (dK_e/dtheta_e) u_e,
  K_ff lambda_f = (dJ/du)_f, lambda = 0 on Dirichlet DOFs.
dC_e/dtheta_e is taken by the complex-step derivative of the tensor rotation
(Im C(theta + i h) / h, exact to rounding), dK_e/dtheta_e = element stiffness
with dC in place of C (the element stiffness is linear in C), and dJ/du by the
chain rule through the (linear) centre-stress map.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem

H_CS = 1e-30


def dC_dtheta(mesh, e):
    """dC_e/dtheta_e by complex step on R = R_l(psi + theta) R_r(phi)."""
    lam = mesh.lam
    base = fem.material_C(lam.materials[mesh.mat_of_elem[e]])
    phi = np.radians(lam.layer_angle_deg[mesh.layer_of_elem[e]])
    a = mesh.psi[e] + mesh.theta[e] + 1j * H_CS
    c, s = np.cos(a), np.sin(a)
    Ry = np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=complex)
    R = Ry @ fem.rot_normal(phi).astype(complex)
    T = fem.voigt_to_tensor(base).astype(complex)
    Tr = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, T, optimize=True)
    return np.imag(_voigt_c(Tr)) / H_CS


def _voigt_c(T):
    C = np.zeros((6, 6), dtype=complex)
    for I, (i, j) in enumerate(fem.VOIGT):
        for J, (k, l) in enumerate(fem.VOIGT):
            C[I, J] = T[i, j, k, l]
    return C


def centre_s33_rows(mesh, e):
    """l_e with s33_e = l_e . u_e (81 entries) and the Voigt weights wv (s33 = wv . sigma)."""
    N, dN = fem.q2_shape(0.0, 0.0, 0.0)
    Xe = mesh.X[mesh.conn[e]]
    J = Xe.T @ dN
    B = fem.strain_B(dN @ np.linalg.inv(J))
    Rf = fem.rot_width(mesh.psi[e])
    wv = np.array([Rf[i, 2] * Rf[j, 2] * (1 if i == j else 2) for i, j in fem.VOIGT])
    return B.T @ (mesh.C[e].T @ wv), wv, B


def objective(mesh, u, mask, p):
    s33, _ = fem.stress_slr(mesh, u)
    return float(np.sum(s33[mask] ** p) ** (1.0 / p)), s33


def gradient(system, mask, p, u=None):
    """Adjoint gradient dJ/dtheta (all elements) of J = ||s33[mask]||_p, direct solves."""
    mesh = system.mesh
    if u is None:
        u = system.direct()
    J, s33 = objective(mesh, u, mask, p)
    w = np.zeros(mesh.n_elem)
    w[mask] = J ** (1.0 - p) * s33[mask] ** (p - 1)
    dJdu = np.zeros(mesh.n_dof)
    explicit = np.zeros(mesh.n_elem)
    for e in np.nonzero(w)[0]:
        l, wv, B = centre_s33_rows(mesh, e)
        d = fem.element_dofs(mesh.conn[e])
        dJdu[d] += w[e] * l
        explicit[e] = w[e] * wv @ dC_dtheta(mesh, e) @ (B @ u[d])
    lam = np.zeros(mesh.n_dof)
    lam[system.free] = spla.splu(system.Kff.tocsc()).solve(dJdu[system.free])
    grad = explicit.copy()
    for e in range(mesh.n_elem):
        if mesh.is_resin[e]:
            continue                                  # isotropic: C does not depend on theta
        dK = fem.element_stiffness(mesh.X[mesh.conn[e]], dC_dtheta(mesh, e))
        d = fem.element_dofs(mesh.conn[e])
        grad[e] -= lam[d] @ dK @ u[d]
    return J, grad, u


def objective_at(lam_spec, theta, mask, p):
    """J for a perturbed misalignment field (fresh mesh + direct solve)."""
    lam_spec.theta = theta.reshape(lam_spec.nz, lam_spec.ny, lam_spec.nx)
    mesh = fem.Mesh(lam_spec)
    u = fem.System(mesh).direct()
    return objective(mesh, u, mask, p)[0]

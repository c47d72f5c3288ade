"""Oracle 20-node serendipity hexahedron (the element the paper's own code uses,
Section 2.1: full 3x3x3 Gauss integration) on the same structured laminates.

Test infrastructure only (see the package docstring); plain FP64 NumPy/SciPy.
The CUDA library builds the triquadratic Q2 element instead; this module
pins the serendipity element against closed forms so that a later GPU
version has its oracle.

Element: 8 corner nodes and 12 edge-midpoint nodes of the reference cube
[-1, 1]^3.  Shape functions (the standard serendipity family):
  corner (xi_a, eta_a, zeta_a in {-1, 1}):
      N = 1/8 (1 + xi xi_a)(1 + eta eta_a)(1 + zeta zeta_a)(xi xi_a + eta eta_a + zeta zeta_a - 2)
  edge midpoint with xi_a = 0 (and likewise for eta_a = 0, zeta_a = 0):
      N = 1/4 (1 - xi^2)(1 + eta eta_a)(1 + zeta zeta_a)
The space holds every quadratic polynomial (and some cubic terms), so on
box-shaped elements quadratic displacement fields are exact.

Mesh: the vertices and edge midpoints of the structured laminate grid, i.e.
the Q2 grid nodes (ix, iy, iz) with at most one odd index; the geometry map,
materials, rotations and loads are those of oracle.fem.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem

# reference coordinates of the 20 nodes: corners first, then edge midpoints
_REF = np.array([(x, y, z) for z in (-1, 1) for y in (-1, 1) for x in (-1, 1)]
                + [(0, y, z) for z in (-1, 1) for y in (-1, 1)]
                + [(x, 0, z) for z in (-1, 1) for x in (-1, 1)]
                + [(x, y, 0) for y in (-1, 1) for x in (-1, 1)], dtype=np.float64)


def shape20(xi, eta, zeta):
    """N (20,) and reference gradients dN (20, 3) at one point."""
    N = np.zeros(20)
    dN = np.zeros((20, 3))
    p = np.array([xi, eta, zeta])
    for a, r in enumerate(_REF):
        if a < 8:
            f = 1.0 + p * r                     # (1 + xi xi_a), ...
            s = p @ r - 2.0
            N[a] = 0.125 * f[0] * f[1] * f[2] * s
            for d in range(3):
                others = np.prod([f[e] for e in range(3) if e != d])
                dN[a, d] = 0.125 * (r[d] * others * s + f[0] * f[1] * f[2] * r[d])
        else:
            d0 = int(np.flatnonzero(r == 0)[0])  # the direction along the edge
            g = 1.0 + p * r
            g[d0] = 1.0 - p[d0] ** 2
            N[a] = 0.25 * g[0] * g[1] * g[2]
            for d in range(3):
                dg = -2.0 * p[d0] if d == d0 else r[d]
                dN[a, d] = 0.25 * dg * np.prod([g[e] for e in range(3) if e != d])
    return N, dN


_GP, _GW = fem.gauss_points_3d()
_SHAPES = [shape20(*q) for q in _GP]


def strain_B20(dNdx):
    """6 x 60 engineering-strain matrix (rows 11, 22, 33, 23, 13, 12)."""
    dx, dy, dz = dNdx[:, 0], dNdx[:, 1], dNdx[:, 2]
    B = np.zeros((6, 60))
    B[0, 0::3] = dx
    B[1, 1::3] = dy
    B[2, 2::3] = dz
    B[3, 1::3], B[3, 2::3] = dz, dy
    B[4, 0::3], B[4, 2::3] = dz, dx
    B[5, 0::3], B[5, 1::3] = dy, dx
    return B


def element_stiffness20(Xe, C):
    """K_e = sum_q w_q |J_q| B_q^T C B_q over the 27 Gauss points (full integration)."""
    Ke = np.zeros((60, 60))
    for (N, dN), w in zip(_SHAPES, _GW):
        J = Xe.T @ dN
        dNdx = dN @ np.linalg.inv(J)
        B = strain_B20(dNdx)
        Ke += w * np.linalg.det(J) * (B.T @ C @ B)
    return Ke


class Mesh20:
    """Serendipity mesh of a laminate: compact node numbering over the Q2 grid
    nodes with at most one odd index, 20-node connectivity, per-element C
    (from oracle.fem.Mesh, whose geometry and materials it shares)."""

    def __init__(self, lam):
        q2 = fem.Mesh(lam)
        self.q2 = q2
        NX, NY, NZ = q2.NX, q2.NY, q2.NZ
        iz, iy, ix = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
        odd = (ix % 2) + (iy % 2) + (iz % 2)
        keep = (odd <= 1).ravel()                  # q2 node order n = ix + NX (iy + NY iz)
        self.q2_of = np.flatnonzero(keep)          # serendipity node -> q2 node
        self.of_q2 = -np.ones(q2.n_nodes, dtype=np.int64)
        self.of_q2[self.q2_of] = np.arange(self.q2_of.size)
        self.X = q2.X[self.q2_of]
        self.n_nodes = self.q2_of.size
        self.n_dof = 3 * self.n_nodes
        self.n_elem = q2.n_elem
        ex, ey, ez = q2.eijk[:, 0], q2.eijk[:, 1], q2.eijk[:, 2]
        conn = np.zeros((self.n_elem, 20), dtype=np.int64)
        for a, r in enumerate(_REF):
            i, j, k = (r + 1).astype(int)          # 0, 1, 2 along each axis
            qn = (2 * ex + i) + NX * ((2 * ey + j) + NY * (2 * ez + k))
            conn[:, a] = self.of_q2[qn]
        assert (conn >= 0).all()
        self.conn = conn
        self.C = q2.C

    def assemble_K(self):
        rows, cols, vals = [], [], []
        for e in range(self.n_elem):
            Ke = element_stiffness20(self.X[self.conn[e]], self.C[e])
            d = (3 * self.conn[e][:, None] + np.arange(3)[None, :]).ravel()
            rows.append(np.repeat(d, 60))
            cols.append(np.tile(d, 60))
            vals.append(Ke.ravel())
        K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.n_dof, self.n_dof))
        return 0.5 * (K + K.T)


def solve_dirichlet(mesh, K, f, dir_dof, dir_val):
    """u with u[dir_dof] = dir_val and (K u - f)[free] = 0, by a sparse direct solve."""
    u = np.zeros(mesh.n_dof)
    u[dir_dof] = dir_val
    free = np.setdiff1d(np.arange(mesh.n_dof), dir_dof)
    rhs = f[free] - K[free][:, dir_dof] @ np.asarray(dir_val)
    u[free] = spla.spsolve(K[free][:, free].tocsc(), rhs)
    return u


def traction_load20(mesh, face, t):
    """Consistent nodal loads of a uniform traction t (MPa) on one box face of
    a serendipity mesh: f_a = int_face N_a t dA by the 3x3 Gauss rule on every
    element face lying on `face` (faces numbered as in oracle.fem: 0 -s, 1 +s,
    2 -l, 3 +l, 4 -r, 5 +r).  On the face the 20 shape functions reduce to the
    8-node serendipity quadrilateral (the others vanish there)."""
    q2 = mesh.q2
    axis, side = fem.FACE_AXIS[face]
    n_e = (q2.nx, q2.ny, q2.nz)[axis]
    fix = -1.0 if side == 0 else 1.0
    e_fix = 0 if side == 0 else n_e - 1
    g, w = fem.gauss3()
    others = [d for d in range(3) if d != axis]
    tv = np.asarray(t, dtype=np.float64)
    f = np.zeros(mesh.n_dof)
    for e in np.nonzero(q2.eijk[:, axis] == e_fix)[0]:
        Xe = mesh.X[mesh.conn[e]]
        d = (3 * mesh.conn[e][:, None] + np.arange(3)[None, :]).ravel()
        for i, a in enumerate(g):
            for j, b in enumerate(g):
                p = [0.0, 0.0, 0.0]
                p[axis] = fix
                p[others[0]] = a
                p[others[1]] = b
                N, dN = shape20(*p)
                J = Xe.T @ dN
                dA = np.linalg.norm(np.cross(J[:, others[0]], J[:, others[1]]))
                f[d] += w[i] * w[j] * dA * np.kron(N, tv)
    return f


def stress_slr20(mesh, u):
    """sigma_33 = sigma_rr and tau_13 = tau_rs at every element centre of a
    serendipity mesh (u in its own numbering): sigma = C_e eps(u) with the
    20-node gradients at xi = 0 and the 20-node geometry map, rotated into the
    local (s, l, r) frame as in oracle.fem.stress_slr."""
    _, dN = shape20(0.0, 0.0, 0.0)
    q2 = mesh.q2
    s33 = np.zeros(mesh.n_elem)
    t13 = np.zeros(mesh.n_elem)
    for e in range(mesh.n_elem):
        Xe = mesh.X[mesh.conn[e]]
        J = Xe.T @ dN
        dNdx = dN @ np.linalg.inv(J)
        d = (3 * mesh.conn[e][:, None] + np.arange(3)[None, :]).ravel()
        sv = mesh.C[e] @ (strain_B20(dNdx) @ u[d])
        S = np.zeros((3, 3))
        for I, (i, j) in enumerate(fem.VOIGT):
            S[i, j] = S[j, i] = sv[I]
        Rf = fem.rot_width(q2.psi[e])
        Sl = Rf.T @ S @ Rf
        s33[e] = Sl[2, 2]
        t13[e] = Sl[0, 2]
    return s33, t13

"""Oracle finite-element layer: Q2 hexahedra for 3D anisotropic linear elasticity.

Test infrastructure only (see the package docstring).  Plain FP64 NumPy/SciPy.

Paper passages followed:
  * Section 2.1: standard anisotropic 3D linear elasticity with a general
    stiffness tensor; quadratic hexahedra with full integration (Section 2.1
    describes the 20-node serendipity element; this build uses the 27-node
    triquadratic Q2 hexahedron with 3x3x3 Gauss points, the full rule);
  * Section 2.2, Table 1: orthotropic ply and isotropic resin constants,
    ply angles about the laminate normal;
  * Section 2.3, Eq. (eq-1): K u = f, K sparse and symmetric;
  * Section 3, the map after Eq. (eq-f): curved corner geometry
    x = L + r sin(pi s/2), y = l, z = r cos(pi s/2).

Readings where the paper is silent:
  * Voigt order (11, 22, 33, 23, 13, 12) with engineering shear strains;
  * ply angle phi rotates about the laminate normal r, misalignment theta about
    the width axis l, then the curved frame rotates about l by the arc angle at
    the element centre: R = R_l(psi) R_l(theta) R_r(phi); C_e is constant per
    element;
  * the curved map's s in [0,1] spans the 90-degree arc, limbs of length L are
    appended tangentially (t in [-1,0] and [1,2]);
  * stresses are recovered at the element centre and rotated into (s, l, r).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]

# --------------------------------------------------------------------------
# 1D quadratic Lagrange basis on {-1, 0, 1} and the 3-point Gauss rule.
# --------------------------------------------------------------------------


def lagrange1(xi):
    """Values of the three quadratic Lagrange polynomials at xi (nodes -1, 0, 1)."""
    xi = np.asarray(xi, dtype=np.float64)
    return np.stack([0.5 * xi * (xi - 1.0), 1.0 - xi * xi, 0.5 * xi * (xi + 1.0)], axis=-1)


def dlagrange1(xi):
    xi = np.asarray(xi, dtype=np.float64)
    return np.stack([xi - 0.5, -2.0 * xi, xi + 0.5], axis=-1)


def gauss3():
    """3-point Gauss-Legendre rule on [-1, 1] (exact to degree 5)."""
    a = math.sqrt(3.0 / 5.0)
    return np.array([-a, 0.0, a]), np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def q2_shape(xi, eta, zeta):
    """27 Q2 shape functions and reference gradients at one point.

    Local node a = i + 3 j + 9 k sits at reference coordinates (i-1, j-1, k-1).
    Returns N (27,) and dN (27, 3) with dN[a, d] = dN_a / dxi_d.
    """
    Nx, Ny, Nz = lagrange1(xi), lagrange1(eta), lagrange1(zeta)
    Dx, Dy, Dz = dlagrange1(xi), dlagrange1(eta), dlagrange1(zeta)
    N = np.zeros(27)
    dN = np.zeros((27, 3))
    for k in range(3):
        for j in range(3):
            for i in range(3):
                a = i + 3 * j + 9 * k
                N[a] = Nx[i] * Ny[j] * Nz[k]
                dN[a, 0] = Dx[i] * Ny[j] * Nz[k]
                dN[a, 1] = Nx[i] * Dy[j] * Nz[k]
                dN[a, 2] = Nx[i] * Ny[j] * Dz[k]
    return N, dN


def gauss_points_3d():
    g, w = gauss3()
    pts, wts = [], []
    for k in range(3):
        for j in range(3):
            for i in range(3):
                pts.append((g[i], g[j], g[k]))
                wts.append(w[i] * w[j] * w[k])
    return np.array(pts), np.array(wts)


# --------------------------------------------------------------------------
# Materials (Table 1) and rotations.
# --------------------------------------------------------------------------


def orthotropic_C(E1, E2, E3, G12, G13, G23, nu12, nu13, nu23, **_):
    """6x6 stiffness of an orthotropic material from its engineering constants.

    Compliance with nu_ij = -eps_j / eps_i under uniaxial stress i, so
    S_ij = -nu_ij / E_i (symmetric since nu_ji = nu_ij E_j / E_i); C = S^{-1}.
    """
    S = np.zeros((6, 6))
    S[0, 0], S[1, 1], S[2, 2] = 1.0 / E1, 1.0 / E2, 1.0 / E3
    S[0, 1] = S[1, 0] = -nu12 / E1
    S[0, 2] = S[2, 0] = -nu13 / E1
    S[1, 2] = S[2, 1] = -nu23 / E2
    S[3, 3], S[4, 4], S[5, 5] = 1.0 / G23, 1.0 / G13, 1.0 / G12
    return np.linalg.inv(S)


def isotropic_C(E, nu, **_):
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    C[[0, 1, 2], [0, 1, 2]] += 2.0 * mu
    C[[3, 4, 5], [3, 4, 5]] = mu
    return C


def material_C(m):
    return orthotropic_C(**m) if m["kind"] == "ortho" else isotropic_C(**m)


def voigt_to_tensor(C):
    T = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, l) in enumerate(VOIGT):
            v = C[I, J]
            for a, b in ((i, j), (j, i)):
                for c, d in ((k, l), (l, k)):
                    T[a, b, c, d] = v
    return T


def tensor_to_voigt(T):
    C = np.zeros((6, 6))
    for I, (i, j) in enumerate(VOIGT):
        for J, (k, l) in enumerate(VOIGT):
            C[I, J] = T[i, j, k, l]
    return C


def rot_normal(phi):
    """Rotation by phi about the laminate normal (the r / z axis)."""
    c, s = math.cos(phi), math.sin(phi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_width(a):
    """Rotation by a about the width axis (l / y); maps e_s to (cos a, 0, -sin a)."""
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rotate_C(C, R):
    """C'_{ijkl} = R_ia R_jb R_kc R_ld C_abcd, R mapping material axes to global axes."""
    T = voigt_to_tensor(C)
    Tr = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, T, optimize=True)
    return tensor_to_voigt(Tr)


# --------------------------------------------------------------------------
# Mesh geometry.
# --------------------------------------------------------------------------


def q2_node_params(v):
    """Q2 node parameters along one axis: vertices at even, midpoints at odd indices."""
    v = np.asarray(v, dtype=np.float64)
    out = np.empty(2 * len(v) - 1)
    out[0::2] = v
    out[1::2] = 0.5 * (v[:-1] + v[1:])
    return out


def rv_vertices(lam):
    out = [0.0]
    base = 0.0
    for n, h in zip(lam.layer_nel, lam.layer_thick):
        for i in range(n):
            out.append(base + h * (i + 1) / n)
        base += h
    return np.asarray(out)


def frame_angle(lam, t):
    """Arc angle psi of the local (s, l, r) frame at parametric coordinate t."""
    if lam.geometry == 0:
        return np.zeros_like(np.asarray(t, dtype=np.float64))
    pe = math.radians(lam.arc_deg)
    return np.clip(np.asarray(t, dtype=np.float64), 0.0, 1.0) * pe


def map_point(lam, t, l, depth):
    """Physical position of parametric (t, l, depth); Section 3 curved map."""
    t = np.asarray(t, dtype=np.float64)
    l = np.asarray(l, dtype=np.float64)
    depth = np.asarray(depth, dtype=np.float64)
    if lam.geometry == 0:
        return np.stack(np.broadcast_arrays(t, l, depth), axis=-1)
    L = lam.limb_L
    r = lam.R_inner + depth
    pe = math.radians(lam.arc_deg)
    psi = np.clip(t, 0.0, 1.0) * pe
    x = L + r * np.sin(psi)
    z = r * np.cos(psi)
    # straight limbs appended along the tangent (cos psi, 0, -sin psi)
    ext = np.where(t < 0.0, t * L, np.where(t > 1.0, (t - 1.0) * L, 0.0))
    x = x + ext * np.cos(psi)
    z = z - ext * np.sin(psi)
    return np.stack(np.broadcast_arrays(x, l, z), axis=-1)


class Mesh:
    """Structured Q2 mesh of a laminate: nodes, connectivity, per-element C."""

    def __init__(self, lam):
        self.lam = lam
        self.nx, self.ny, self.nz = lam.nx, lam.ny, lam.nz
        self.NX, self.NY, self.NZ = 2 * self.nx + 1, 2 * self.ny + 1, 2 * self.nz + 1
        self.n_nodes = self.NX * self.NY * self.NZ
        self.n_dof = 3 * self.n_nodes
        self.n_elem = self.nx * self.ny * self.nz
        tn = q2_node_params(lam.sv)
        ln = q2_node_params(lam.lv)
        rn = q2_node_params(rv_vertices(lam))
        T, Lg, R = np.meshgrid(tn, ln, rn, indexing="ij")      # (NX, NY, NZ)
        dr = getattr(lam, "node_dr", None)
        if dr is not None:
            # geometric wrinkle (Section 3, Eq. eq-wrinkle): r^ = r + f, before the map
            R = R + np.asarray(dr).reshape(self.NZ, self.NY, self.NX).transpose(2, 1, 0)
        X = map_point(lam, T, Lg, R)
        # node n = ix + NX*(iy + NY*iz)
        self.X = X.transpose(2, 1, 0, 3).reshape(-1, 3)
        ex, ey, ez = np.meshgrid(np.arange(self.nx), np.arange(self.ny), np.arange(self.nz),
                                 indexing="ij")
        ex, ey, ez = (a.transpose(2, 1, 0).ravel() for a in (ex, ey, ez))   # e = ex + nx*(ey + ny*ez)
        self.eijk = np.stack([ex, ey, ez], axis=1)
        conn = np.zeros((self.n_elem, 27), dtype=np.int64)
        for k in range(3):
            for j in range(3):
                for i in range(3):
                    conn[:, i + 3 * j + 9 * k] = (2 * ex + i) + self.NX * ((2 * ey + j) + self.NY * (2 * ez + k))
        self.conn = conn
        self.layer_of_elem = np.repeat(np.arange(len(lam.layer_nel)), lam.layer_nel)[ez]
        self.mat_of_elem = np.asarray(lam.layer_mat)[self.layer_of_elem]
        if getattr(lam, "elem_mat", None) is not None:
            self.mat_of_elem = np.asarray(lam.elem_mat).reshape(-1).astype(np.int64)
        tc = 0.5 * (np.asarray(lam.sv)[ex] + np.asarray(lam.sv)[ex + 1])
        self.psi = frame_angle(lam, tc)
        theta = np.zeros(self.n_elem) if lam.theta is None else np.asarray(lam.theta).reshape(-1)
        self.theta = theta
        base_C = [material_C(m) for m in lam.materials]
        phi = np.radians(np.asarray(lam.layer_angle_deg, dtype=np.float64))[self.layer_of_elem]
        self.C = np.zeros((self.n_elem, 6, 6))
        self.R = np.zeros((self.n_elem, 3, 3))
        cache = {}
        for e in range(self.n_elem):
            R = rot_width(self.psi[e]) @ rot_width(theta[e]) @ rot_normal(phi[e])
            key = (self.mat_of_elem[e], round(self.psi[e] + theta[e], 15), round(phi[e], 15))
            if key not in cache:
                cache[key] = rotate_C(base_C[self.mat_of_elem[e]], R)
            self.C[e] = cache[key]
            self.R[e] = R
        self.is_resin = np.array([lam.materials[m]["kind"] == "iso" for m in self.mat_of_elem])


# --------------------------------------------------------------------------
# Element stiffness and assembly (Eq. eq-1).
# --------------------------------------------------------------------------


def strain_B(dNdx):
    """6 x 81 engineering-strain matrix from physical shape gradients (27, 3).

    Rows (eps11, eps22, eps33, gamma23, gamma13, gamma12); column 3a+c is
    displacement component c of node a.
    """
    dx, dy, dz = dNdx[:, 0], dNdx[:, 1], dNdx[:, 2]
    B = np.zeros((6, 81))
    B[0, 0::3] = dx
    B[1, 1::3] = dy
    B[2, 2::3] = dz
    B[3, 1::3], B[3, 2::3] = dz, dy
    B[4, 0::3], B[4, 2::3] = dz, dx
    B[5, 0::3], B[5, 1::3] = dy, dx
    return B


_GP, _GW = gauss_points_3d()
_SHAPES = [q2_shape(*p) for p in _GP]


def element_stiffness(Xe, C):
    """K_e = sum_q w_q |J_q| B_q^T C B_q over the 27 Gauss points (full integration)."""
    Ke = np.zeros((81, 81))
    for (N, dN), w in zip(_SHAPES, _GW):
        J = Xe.T @ dN                       # J[i, j] = dx_i / dxi_j
        detJ = np.linalg.det(J)
        dNdx = dN @ np.linalg.inv(J)        # dN_a/dx_i
        B = strain_B(dNdx)
        Ke += w * detJ * (B.T @ C @ B)
    return Ke


def element_dofs(conn_e):
    return (3 * np.asarray(conn_e)[:, None] + np.arange(3)[None, :]).ravel()


def assemble_K(mesh, elems=None):
    """Global (or partial, over `elems`) stiffness as CSR, all DOFs."""
    if elems is None:
        elems = range(mesh.n_elem)
    rows, cols, vals = [], [], []
    for e in elems:
        Ke = element_stiffness(mesh.X[mesh.conn[e]], mesh.C[e])
        d = element_dofs(mesh.conn[e])
        rows.append(np.repeat(d, 81))
        cols.append(np.tile(d, 81))
        vals.append(Ke.ravel())
    if not rows:
        return sp.csr_matrix((mesh.n_dof, mesh.n_dof))
    K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.n_dof, mesh.n_dof)).tocsr()
    K.sum_duplicates()
    return K


# --------------------------------------------------------------------------
# Loads and Dirichlet data.
# --------------------------------------------------------------------------

FACE_AXIS = {0: (0, 0), 1: (0, 1), 2: (1, 0), 3: (1, 1), 4: (2, 0), 5: (2, 1)}


def traction_load(mesh, face, t):
    """Consistent nodal loads of a surface traction on one box face.

    f_a = int_face N_a t dA with the 3x3 Gauss rule on every boundary face of
    the elements touching `face`.  `t` is a 3-vector (MPa) or a callable of
    the physical position returning one.
    """
    axis, side = FACE_AXIS[face]
    n_e = (mesh.nx, mesh.ny, mesh.nz)[axis]
    fix = -1.0 if side == 0 else 1.0
    e_fix = 0 if side == 0 else n_e - 1
    g, w = gauss3()
    f = np.zeros(mesh.n_dof)
    others = [d for d in range(3) if d != axis]
    for e in np.nonzero(mesh.eijk[:, axis] == e_fix)[0]:
        Xe = mesh.X[mesh.conn[e]]
        for i, a in enumerate(g):
            for j, b in enumerate(g):
                p = [0.0, 0.0, 0.0]
                p[axis] = fix
                p[others[0]] = a
                p[others[1]] = b
                N, dN = q2_shape(*p)
                J = Xe.T @ dN
                dA = np.linalg.norm(np.cross(J[:, others[0]], J[:, others[1]]))
                x = N @ Xe
                tv = np.asarray(t(x) if callable(t) else t, dtype=np.float64)
                d = element_dofs(mesh.conn[e])
                f[d] += w[i] * w[j] * dA * np.kron(N, tv)
    return f


def load_vector(mesh):
    f = np.zeros(mesh.n_dof)
    for face, t in mesh.lam.traction:
        f += traction_load(mesh, face, t)
    return f


class System:
    """K u = f with the Dirichlet DOFs eliminated (lifted into the right-hand side)."""

    def __init__(self, mesh, K=None, f=None, dir_dof=None, dir_val=None):
        self.mesh = mesh
        self.K = assemble_K(mesh) if K is None else K
        self.f = load_vector(mesh) if f is None else f
        lam = mesh.lam
        self.dir_dof = np.asarray(lam.dir_dof if dir_dof is None else dir_dof, dtype=np.int64)
        self.dir_val = np.asarray(lam.dir_val if dir_val is None else dir_val, dtype=np.float64)
        n = mesh.n_dof
        self.is_dir = np.zeros(n, dtype=bool)
        self.is_dir[self.dir_dof] = True
        self.free = np.nonzero(~self.is_dir)[0]
        self.u_dir = np.zeros(n)
        self.u_dir[self.dir_dof] = self.dir_val
        self.Kff = self.K[self.free][:, self.free].tocsr()
        self.ff = (self.f - self.K @ self.u_dir)[self.free]

    def full(self, uf):
        u = self.u_dir.copy()
        u[self.free] = uf
        return u

    def direct(self):
        """Exact-result definition u = K^{-1} f (sparse LU)."""
        uf = spla.splu(self.Kff.tocsc()).solve(self.ff)
        return self.full(uf)


def periodic_width_direct(mesh, dir_dof, dir_val, f=None, K=None):
    """Direct solve with periodic width conditions, u(s, 0, r) = u(s, W, r), as in
    the paper's 39-ply study (Section 3).  Every node of the last width plane
    (iy = NY - 1) is identified with its partner on the first (iy = 0): with A
    the n_dof x n_master selection matrix, K_p = A^T K A and f_p = A^T f;
    Dirichlet DOFs are given in full-mesh numbering (a DOF on the last plane
    stands for its partner).  Returns the full displacement (both planes carry
    the same values)."""
    n = mesh.n_dof
    K = assemble_K(mesh) if K is None else K
    f = load_vector(mesh) if f is None else f
    node = np.arange(mesh.n_nodes)
    iy = (node // mesh.NX) % mesh.NY
    rep_node = np.where(iy == mesh.NY - 1, node - (mesh.NY - 1) * mesh.NX, node)
    rep = (3 * rep_node[:, None] + np.arange(3)[None, :]).ravel()       # DOF -> its master DOF
    masters = np.unique(rep)
    col = -np.ones(n, dtype=np.int64)
    col[masters] = np.arange(masters.size)
    A = sp.csr_matrix((np.ones(n), (np.arange(n), col[rep])), shape=(n, masters.size))
    Kp = (A.T @ K @ A).tocsr()
    fp = A.T @ f
    # a DOF on the last plane and its partner may both be listed: keep each master once
    d, first = np.unique(col[rep[np.asarray(dir_dof, dtype=np.int64)]], return_index=True)
    up = np.zeros(masters.size)
    up[d] = np.asarray(dir_val, dtype=np.float64)[first]
    free = np.setdiff1d(np.arange(masters.size), d)
    rhs = fp[free] - Kp[free][:, d] @ up[d]
    up[free] = spla.splu(Kp[free][:, free].tocsc()).solve(rhs)
    return A @ up


# --------------------------------------------------------------------------
# Stress recovery (Section 2.2 notation sigma_r, tau_rs; Eq. eq-Camanho uses them).
# --------------------------------------------------------------------------


def element_stress_centre(mesh, u):
    """Stress tensor (global axes) at every element centre, sigma = C_e eps(u)."""
    N, dN = q2_shape(0.0, 0.0, 0.0)
    out = np.zeros((mesh.n_elem, 3, 3))
    for e in range(mesh.n_elem):
        Xe = mesh.X[mesh.conn[e]]
        J = Xe.T @ dN
        dNdx = dN @ np.linalg.inv(J)
        ue = u[element_dofs(mesh.conn[e])]
        eps = strain_B(dNdx) @ ue
        sv = mesh.C[e] @ eps
        S = np.zeros((3, 3))
        for I, (i, j) in enumerate(VOIGT):
            S[i, j] = S[j, i] = sv[I]
        out[e] = S
    return out


def stress_slr(mesh, u):
    """sigma_33 = sigma_rr and tau_13 = tau_rs in the local (s, l, r) frame, per element."""
    S = element_stress_centre(mesh, u)
    s33 = np.zeros(mesh.n_elem)
    t13 = np.zeros(mesh.n_elem)
    for e in range(mesh.n_elem):
        Rf = rot_width(mesh.psi[e])           # columns: e_s, e_l, e_r in global axes
        Sl = Rf.T @ S[e] @ Rf
        s33[e] = Sl[2, 2]
        t13[e] = Sl[0, 2]
    return s33, t13


def failure_index(mesh, u, s33=61.0, s13=97.0):
    """Quadratic damage-onset criterion (Section 3.2, Eq. eq-Camanho) per element.

    F = sqrt((max(sigma_r, 0)/s33)^2 + (tau_rs/s13)^2 + (tau_rl/s13)^2) from the
    centre stress in the local (s, l, r) frame, evaluated in the isotropic
    resin interfaces only (0 elsewhere); allowables s33 = 61 MPa, s13 = 97 MPa.
    """
    S = element_stress_centre(mesh, u)
    F = np.zeros(mesh.n_elem)
    for e in np.nonzero(mesh.is_resin)[0]:
        Rf = rot_width(mesh.psi[e])
        Sl = Rf.T @ S[e] @ Rf
        F[e] = np.sqrt((max(Sl[2, 2], 0.0) / s33) ** 2 + (Sl[0, 2] / s13) ** 2 + (Sl[1, 2] / s13) ** 2)
    return F

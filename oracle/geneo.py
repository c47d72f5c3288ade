"""Oracle GenEO two-level overlapping Schwarz and PCG (Section 2.3).

Test infrastructure only (see the package docstring).  Plain FP64 SciPy.

What the paper states (Section 2.3, "Efficiency of dune-composites: Robust
iterative solvers", and Fig. domaindecomp / Fig. eig):
  * CG on the preconditioned system P K u = P f (Eq. eq-pre);
  * the mesh is split into overlapping subdomains of roughly equal size
    (overlap of one or two elements);
  * on each subdomain the problem with zero displacement on the artificial
    subdomain boundary is solved by a direct method;
  * a coarse space is built from a few of the lowest-energy eigenmodes of local
    generalised eigenproblems (including the rigid-body modes), glued by a
    partition of unity; the coarse problem is solved by a direct method;
  * two-level additive Schwarz = coarse correction + sum of local solves.

Readings (the paper defers the GenEO details to its reference [geneo2]; this
restates the standard published construction):
  * element boxes from a near-equal split of each index range (the first
    n % p boxes get one extra element), grown by `overlap` element layers;
  * V_j^N = free DOFs of the closed subdomain; artificial-boundary DOFs are
    nodes of the closed subdomain that also belong to an element outside it;
    V_j = V_j^N without them; A_j = K restricted to V_j (Dirichlet matrix);
    A_j^N assembled from the subdomain's elements only, on V_j^N (Neumann);
  * partition of unity Xi_j(i) = 1 / #{k : i in V_k} on V_j, 0 on the
    artificial boundary, so sum_j R_j^T Xi_j R_j = I on the free DOFs;
  * GenEO: A_j^N p = lambda B_j p with B_j = Xi_j A_j^N Xi_j, keep the nev
    smallest lambda; solved through the definite pencil
    B p = mu (A_j^N + sigma B_j) p, lambda = 1/mu - sigma;
  * coarse basis Z = [R_j^T Xi_j p_j^k], K_0 = Z^T K Z, dense Cholesky;
    columns that are linearly dependent on earlier ones (Cholesky pivot of
    K_0 scaled to unit diagonal <= 1e-10, e.g. from two subdomains that
    coincide on a narrow laminate) are left out of Z;
  * M^{-1} = Z K_0^{-1} Z^T + sum_j R_j^T A_j^{-1} R_j (additive);
  * PCG from x_0 = 0, stop when ||r_k||_2 / ||r_0||_2 <= tol.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


def split_range(n, p):
    """Near-equal split of range(n) into p pieces: (start, stop) pairs."""
    q, r = divmod(n, p)
    out, s = [], 0
    for i in range(p):
        size = q + (1 if i < r else 0)
        out.append((s, s + size))
        s += size
    return out


class Subdomain:
    pass


class Decomposition:
    """Overlapping box decomposition, DOF sets and partition of unity."""

    def __init__(self, system, px, py, pz, overlap=1):
        mesh = system.mesh
        self.system, self.mesh = system, mesh
        self.p = (px, py, pz)
        n_e = (mesh.nx, mesh.ny, mesh.nz)
        free_idx = -np.ones(mesh.n_dof, dtype=np.int64)
        free_idx[system.free] = np.arange(system.free.size)
        self.free_idx = free_idx
        ranges = [split_range(n_e[a], self.p[a]) for a in range(3)]
        self.subs = []
        for kz in range(pz):
            for ky in range(py):
                for kx in range(px):
                    s = Subdomain()
                    s.core = [ranges[0][kx], ranges[1][ky], ranges[2][kz]]
                    s.box = [(max(0, a - overlap), min(n_e[d], b + overlap))
                             for d, (a, b) in enumerate(s.core)]
                    self.subs.append(s)
        for s in self.subs:
            (x0, x1), (y0, y1), (z0, z1) = s.box
            e = mesh.eijk
            s.elems = np.nonzero((e[:, 0] >= x0) & (e[:, 0] < x1) & (e[:, 1] >= y0) & (e[:, 1] < y1)
                                 & (e[:, 2] >= z0) & (e[:, 2] < z1))[0]
            ix, iy, iz = np.meshgrid(np.arange(2 * x0, 2 * x1 + 1), np.arange(2 * y0, 2 * y1 + 1),
                                     np.arange(2 * z0, 2 * z1 + 1), indexing="ij")
            ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
            art = np.zeros(ix.size, dtype=bool)
            for c, (a, b), n in ((ix, s.box[0], n_e[0]), (iy, s.box[1], n_e[1]), (iz, s.box[2], n_e[2])):
                art |= (c == 2 * a) & (a > 0)
                art |= (c == 2 * b) & (b < n)
            nodes = ix + mesh.NX * (iy + mesh.NY * iz)
            order = np.argsort(nodes)
            nodes, art = nodes[order], art[order]
            dof = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
            art_dof = np.repeat(art, 3)
            fi = free_idx[dof]
            keep = fi >= 0
            s.VN = fi[keep]                          # free indices of V_j^N
            s.art = art_dof[keep]                    # artificial-boundary flag on V_j^N
            s.V = s.VN[~s.art]                       # free indices of V_j
        nf = system.free.size
        mult = np.zeros(nf)
        for s in self.subs:
            mult[s.V] += 1.0
        if np.any(mult == 0):
            raise ValueError("some free DOF lies in no subdomain interior (overlap must be >= 1)")
        self.mult = mult
        for s in self.subs:
            s.xi = np.where(s.art, 0.0, 1.0 / mult[s.VN])   # Xi_j on V_j^N

    def dirichlet_matrix(self, s):
        """A_j = R_j K R_j^T on V_j."""
        return self.system.Kff[s.V][:, s.V].tocsc()

    def neumann_matrix(self, s):
        """A_j^N assembled from the subdomain's elements only, restricted to V_j^N."""
        KN = fem.assemble_K(self.mesh, s.elems)
        free = self.system.free
        return KN[free][:, free][s.VN][:, s.VN].tocsc()


def geneo_eigs(AN, xi, nev, sigma=1e-2, method="arpack"):
    """nev smallest eigenpairs of A^N p = lambda (Xi A^N Xi) p.

    Through the definite pencil B p = mu (A^N + sigma B) p (B = Xi A^N Xi is
    only semi-definite and A^N is singular on floating subdomains); the
    largest mu give the smallest lambda = 1/mu - sigma.  Eigenvectors do not
    depend on sigma.  Returns (lambda ascending, P with columns p_k).
    """
    Xi = sp.diags(xi)
    B = (Xi @ AN @ Xi).tocsc()
    M = (AN + sigma * B).tocsc()
    n = AN.shape[0]
    k = min(nev, n)
    if method == "dense":
        mu, P = sla.eigh(B.toarray(), M.toarray(), subset_by_index=[n - k, n - 1])
    else:
        lu = spla.splu(M)
        Minv = spla.LinearOperator((n, n), matvec=lu.solve, dtype=np.float64)
        mu, P = spla.eigsh(B, k=k, M=M, Minv=Minv, which="LA", tol=1e-13,
                           ncv=min(n, max(4 * k + 1, 40)), maxiter=20000)
    lam = 1.0 / mu - sigma
    order = np.argsort(lam)
    return lam[order], P[:, order]


COARSE_DROP_TOL = 1e-10


def independent_columns(K0, tol=COARSE_DROP_TOL):
    """Columns kept by a Cholesky factorisation of K0 scaled to unit diagonal
    that leaves out every column whose pivot is <= tol in magnitude (a column
    in the span of the earlier ones, or a zero column).  Plain column-by-column
    Cholesky in index order; raises on a negative pivot beyond tol."""
    d = np.diag(K0).astype(float)
    scale = np.zeros_like(d)
    scale[d > 0] = 1.0 / np.sqrt(d[d > 0])
    A = K0 * scale[:, None] * scale[None, :]
    n = A.shape[0]
    L = np.zeros_like(A)
    keep = []
    for j in range(n):
        v = A[j, j] - L[j, :j] @ L[j, :j]
        if abs(v) <= tol:
            continue                      # column j stays out of the factor
        if v < 0.0:
            raise np.linalg.LinAlgError("coarse matrix not positive semi-definite")
        L[j, j] = np.sqrt(v)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
        keep.append(j)
    return np.array(keep, dtype=np.int64)


class GenEO:
    """Two-level additive Schwarz preconditioner with a GenEO coarse space."""

    def __init__(self, dec, nev, coarse=True, eig_method="arpack", sigma=1e-2):
        self.dec = dec
        Kff = dec.system.Kff
        nf = Kff.shape[0]
        self.local = []
        for s in dec.subs:
            self.local.append(spla.splu(dec.dirichlet_matrix(s)))
        self.coarse = coarse
        self.eigvals = []
        self.n_dropped = 0
        if coarse:
            cols, rows, vals = [], [], []
            c = 0
            for s in dec.subs:
                AN = dec.neumann_matrix(s)
                lam, P = geneo_eigs(AN, s.xi, nev, sigma=sigma, method=eig_method)
                self.eigvals.append(lam)
                for k in range(P.shape[1]):
                    v = s.xi * P[:, k]
                    nz = v != 0.0
                    rows.append(s.VN[nz])
                    vals.append(v[nz])
                    cols.append(np.full(int(nz.sum()), c))
                    c += 1
            self.Z = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                   shape=(nf, c))
            K0 = (self.Z.T @ (Kff @ self.Z)).toarray()
            K0 = 0.5 * (K0 + K0.T)
            keep = independent_columns(K0)
            self.n_dropped = c - len(keep)
            self.Z_all = self.Z
            self.Z = self.Z[:, keep]
            self.K0 = K0[np.ix_(keep, keep)]
            self.K0_chol = sla.cho_factor(self.K0, lower=True)

    def apply(self, r):
        """z = Z K_0^{-1} Z^T r + sum_j R_j^T A_j^{-1} R_j r."""
        z = np.zeros_like(r)
        for s, lu in zip(self.dec.subs, self.local):
            z[s.V] += lu.solve(r[s.V])
        if self.coarse:
            y = sla.cho_solve(self.K0_chol, self.Z.T @ r)
            z += self.Z @ y
        return z


def pcg(K, f, M=None, tol=1e-10, max_iter=2000, x0=None):
    """Preconditioned CG (Hestenes-Stiefel, rho = r.z), Section 2.3.

    Stops when ||r_k|| / ||r_0|| <= tol with r_0 = f - K x_0.  Returns
    (x, iterations, list of relative residual norms).
    """
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - K @ x
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    z = r.copy() if M is None else M(r)
    p = z.copy()
    rho = r @ z
    for it in range(1, max_iter + 1):
        q = K @ p
        alpha = rho / (p @ q)
        x += alpha * p
        r -= alpha * q
        rel = np.linalg.norm(r) / r0
        hist.append(rel)
        if rel <= tol:
            return x, it, hist
        z = r.copy() if M is None else M(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return x, max_iter, hist


def solve(lam, nev=None, px=None, py=None, pz=None, overlap=None, tol=None, coarse=True,
          eig_method="arpack", system=None, max_iter=2000):
    """Full oracle solve of a laminate with GenEO-PCG.  Returns (u, iters, hist, precond, system)."""
    if system is None:
        system = fem.System(fem.Mesh(lam))
    dec = Decomposition(system, px or lam.px, py or lam.py, pz or lam.pz,
                        lam.overlap if overlap is None else overlap)
    P = GenEO(dec, nev or lam.nev, coarse=coarse, eig_method=eig_method)
    uf, it, hist = pcg(system.Kff, system.ff, P.apply, tol=tol or lam.tol, max_iter=max_iter)
    return system.full(uf), it, hist, P, system

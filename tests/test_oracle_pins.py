"""Pins for the CPU oracle: closed forms, invariants and brute force (no GPU).

Each test checks the oracle against something other than itself: an exact
elasticity solution that Q2 reproduces to round-off, a property the
mathematics fixes, a textbook routine, or values printed in the paper.
"""
import math
import os

import numpy as np
import pytest
from scipy.linalg import solve as sla_solve

from oracle import fem, geneo
from paper_1707_04228_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def block(nx, ny, layers, sx=1.0, sy=1.0, mats=None, geometry=0, **kw):
    """Laminate spec helper: layers = [(nel, thick, mat, angle_deg)]."""
    nel, th, mat, ang = (list(t) for t in zip(*layers))
    sv = np.linspace(0.0, sx, nx + 1) if np.isscalar(sx) else np.asarray(sx)
    lv = np.linspace(0.0, sy, ny + 1) if np.isscalar(sy) else np.asarray(sy)
    return inputs.Laminate(name="t", geometry=geometry, sv=sv, lv=lv, layer_nel=nel,
                           layer_thick=th, layer_mat=mat, layer_angle_deg=ang,
                           materials=mats or [inputs.PLY_T1, inputs.RESIN_T1], **kw)


def all_boundary_nodes(mesh):
    NX, NY, NZ = mesh.NX, mesh.NY, mesh.NZ
    ix, iy, iz = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    b = (ix == 0) | (ix == NX - 1) | (iy == 0) | (iy == NY - 1) | (iz == 0) | (iz == NZ - 1)
    return np.sort((ix + NX * (iy + NY * iz))[b])


# --------------------------------------------------------------------------- basis


def test_q2_basis_partition_of_unity_and_kronecker():
    rng = np.random.default_rng(0)
    for p in rng.uniform(-1, 1, size=(20, 3)):
        N, dN = fem.q2_shape(*p)
        assert abs(N.sum() - 1.0) < 1e-14
        assert np.abs(dN.sum(axis=0)).max() < 1e-13
    for k in range(3):
        for j in range(3):
            for i in range(3):
                N, _ = fem.q2_shape(i - 1.0, j - 1.0, k - 1.0)
                e = np.zeros(27)
                e[i + 3 * j + 9 * k] = 1.0
                assert np.abs(N - e).max() < 1e-15


def test_gauss3_exact_to_degree5():
    g, w = fem.gauss3()
    for d in range(6):
        exact = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs((w * g ** d).sum() - exact) < 1e-15
    assert abs((w * g ** 6).sum() - 2.0 / 7.0) > 1e-3   # and not beyond


# --------------------------------------------------------------------------- materials


def test_table1_constants_match_paper():
    vals = {}
    for line in open(os.path.join(GOLDEN, "table1_materials.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    p, r = inputs.PLY_T1, inputs.RESIN_T1
    gpa = 1000.0
    assert p["E1"] == vals["E11"] * gpa and p["E2"] == vals["E22"] * gpa and p["E3"] == vals["E33"] * gpa
    assert p["G12"] == vals["G12"] * gpa and p["G13"] == vals["G13"] * gpa and p["G23"] == vals["G23"] * gpa
    assert p["nu12"] == vals["nu12"] and p["nu13"] == vals["nu13"] and p["nu23"] == vals["nu23"]
    assert r["E"] == vals["E_resin"] * gpa and r["nu"] == vals["nu_resin"]


def test_orthotropic_engineering_constants():
    """Uniaxial stress and pure shear recover the defining engineering constants."""
    m = inputs.PLY_T1
    C = fem.orthotropic_C(**m)
    assert np.allclose(C, C.T, rtol=0, atol=1e-9 * np.abs(C).max())
    assert np.linalg.eigvalsh(C).min() > 0
    e = np.linalg.solve(C, [1.0, 0, 0, 0, 0, 0])
    assert np.allclose(e, [1 / m["E1"], -m["nu12"] / m["E1"], -m["nu13"] / m["E1"], 0, 0, 0], rtol=1e-12, atol=1e-20)
    e = np.linalg.solve(C, [0, 1.0, 0, 0, 0, 0])
    assert np.allclose(e, [-m["nu12"] / m["E1"], 1 / m["E2"], -m["nu23"] / m["E2"], 0, 0, 0], rtol=1e-12, atol=1e-20)
    for I, G in ((3, m["G23"]), (4, m["G13"]), (5, m["G12"])):
        s = np.zeros(6)
        s[I] = 1.0
        assert abs(np.linalg.solve(C, s)[I] - 1.0 / G) < 1e-12 / G


def test_isotropic_lame():
    E, nu = 10000.0, 0.35
    C = fem.isotropic_C(E, nu)
    e = np.linalg.solve(C, [1.0, 0, 0, 0, 0, 0])
    assert np.allclose(e[:3], [1 / E, -nu / E, -nu / E], rtol=1e-12)
    assert abs(np.linalg.solve(C, [0, 0, 0, 1.0, 0, 0])[3] - 2 * (1 + nu) / E) < 1e-15


def _energy(C, eps_tensor):
    v = np.array([eps_tensor[i, j] * (1 if i == j else 2) for i, j in fem.VOIGT])
    return v @ C @ v


def test_rotation_preserves_energy_and_composes():
    rng = np.random.default_rng(1)
    C = fem.orthotropic_C(**inputs.PLY_T1)
    for _ in range(5):
        a, b, c = rng.uniform(-math.pi, math.pi, 3)
        R = fem.rot_width(a) @ fem.rot_width(b) @ fem.rot_normal(c)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        Cr = fem.rotate_C(C, R)
        eg = rng.standard_normal((3, 3))
        eg = 0.5 * (eg + eg.T)
        em = R.T @ eg @ R                      # the same strain in material axes
        assert abs(_energy(Cr, eg) - _energy(C, em)) < 1e-10 * abs(_energy(C, em))
        # composing two rotations about the width axis adds the angles
        C1 = fem.rotate_C(fem.rotate_C(C, fem.rot_width(b)), fem.rot_width(a))
        C2 = fem.rotate_C(C, fem.rot_width(a + b))
        assert np.allclose(C1, C2, rtol=0, atol=1e-9 * np.abs(C).max())
    # 90 degrees about the normal swaps the in-plane axes
    C90 = fem.rotate_C(C, fem.rot_normal(math.pi / 2))
    perm = [1, 0, 2, 4, 3, 5]
    assert np.allclose(C90, C[np.ix_(perm, perm)], rtol=0, atol=1e-9 * np.abs(C).max())


# --------------------------------------------------------------------------- element / assembly


def _solve_with_exact_dirichlet(lam, ufun, nodes):
    mesh = fem.Mesh(lam)
    X = mesh.X[nodes]
    U = ufun(X)
    dof = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    sysm = fem.System(mesh, f=np.zeros(mesh.n_dof), dir_dof=dof, dir_val=U.ravel())
    return mesh, sysm.direct()


@pytest.mark.parametrize("curved", [False, True])
def test_patch_test_linear_field_exact(curved):
    """Any linear displacement prescribed on the boundary is reproduced inside (Q2 patch test)."""
    rng = np.random.default_rng(2)
    if curved:
        # the material frame follows the arc, so only an isotropic C is homogeneous here
        lam = block(5, 2, [(2, 0.4, 1, 0.0), (1, 0.05, 1, 0.0)], sx=inputs.graded(5, -1.0, 2.0, 3.0),
                    sy=[0.0, 0.7, 2.0], geometry=1, R_inner=2.0, limb_L=1.5, arc_deg=90.0)
    else:
        lam = block(3, 2, [(3, 1.0, 0, 30.0)], sx=[0.0, 0.5, 2.0, 2.4], sy=[0.0, 1.0, 1.3])
        lam.theta = np.full((3, 2, 3), -0.3)
    A = rng.standard_normal((3, 3)) * 1e-3
    b = rng.standard_normal(3) * 1e-3
    mesh = fem.Mesh(lam)
    nodes = all_boundary_nodes(mesh)
    mesh, u = _solve_with_exact_dirichlet(lam, lambda X: X @ A.T + b, nodes)
    exact = (mesh.X @ A.T + b).ravel()
    assert np.linalg.norm(u - exact) <= 1e-11 * np.linalg.norm(exact)


def test_patch_test_on_wrinkled_curved_mesh():
    """The geometric wrinkle moves nodes inside the Q2 (isoparametric) space:
    a linear field prescribed on the boundary is still reproduced inside."""
    rng = np.random.default_rng(5)
    lam = block(6, 3, [(2, 0.4, 1, 0.0), (2, 0.3, 1, 0.0)], sx=inputs.graded(6, -1.0, 2.0, 3.0),
                sy=[0.0, 0.7, 1.4, 2.0], geometry=1, R_inner=2.0, limb_L=1.5, arc_deg=90.0)
    lam.node_dr, _ = inputs.sech2_wrinkle(lam, 0.04)
    A = rng.standard_normal((3, 3)) * 1e-3
    b = rng.standard_normal(3) * 1e-3
    mesh = fem.Mesh(lam)
    plain = fem.Mesh(block(6, 3, [(2, 0.4, 1, 0.0), (2, 0.3, 1, 0.0)], sx=inputs.graded(6, -1.0, 2.0, 3.0),
                           sy=[0.0, 0.7, 1.4, 2.0], geometry=1, R_inner=2.0, limb_L=1.5, arc_deg=90.0))
    assert np.abs(mesh.X - plain.X).max() > 0.01           # the nodes did move
    nodes = all_boundary_nodes(mesh)
    mesh, u = _solve_with_exact_dirichlet(lam, lambda X: X @ A.T + b, nodes)
    exact = (mesh.X @ A.T + b).ravel()
    assert np.linalg.norm(u - exact) <= 1e-11 * np.linalg.norm(exact)


def test_wrinkle_fibre_angle_follows_the_deformed_plies():
    """On a flat plate the misalignment returned with the wrinkle equals minus the
    slope of the deformed ply surfaces measured on the oracle mesh (central
    differences of the element-centre node heights along x), and a zero
    amplitude leaves the mesh unchanged."""
    lam = block(40, 4, [(6, 1.2, 0, 0.0)], sx=8.0, sy=4.0)
    lam.node_dr, theta = inputs.sech2_wrinkle(lam, 0.1, b1=0.3)
    mesh = fem.Mesh(lam)
    Z = mesh.X[:, 2].reshape(mesh.NZ, mesh.NY, mesh.NX)
    X = mesh.X[:, 0].reshape(mesh.NZ, mesh.NY, mesh.NX)
    # element centres are the odd nodes; their neighbours along x are the even nodes
    zc = Z[1::2, 1::2, :]
    slope = (zc[:, :, 2::2] - zc[:, :, 0:-1:2]) / (X[1::2, 1::2, 2::2] - X[1::2, 1::2, 0:-1:2])
    assert np.abs(theta).max() > np.radians(2.0)
    # central differences over one element length: O(h^2), about 1% here
    assert np.abs(theta + np.arctan(slope)).max() <= 0.03 * np.abs(theta).max()
    flat = fem.Mesh(block(40, 4, [(6, 1.2, 0, 0.0)], sx=8.0, sy=4.0))
    lam0 = block(40, 4, [(6, 1.2, 0, 0.0)], sx=8.0, sy=4.0)
    lam0.node_dr, th0 = inputs.sech2_wrinkle(lam0, 0.0)
    assert np.array_equal(fem.Mesh(lam0).X, flat.X) and np.all(th0 == 0.0)


def test_symmetry_and_rigid_body_null_space():
    lam = block(2, 2, [(1, 0.3, 0, 45.0), (1, 0.1, 1, 0.0)], sx=[-0.5, 0.3, 1.0], sy=1.0,
                geometry=1, R_inner=1.0, limb_L=1.0)
    lam.theta = np.full((2, 2, 2), 0.1)
    mesh = fem.Mesh(lam)
    K = fem.assemble_K(mesh).toarray()
    nK = np.abs(K).max()
    assert np.abs(K - K.T).max() <= 1e-13 * nK
    X = mesh.X
    modes = []
    for d in range(3):
        m = np.zeros_like(X)
        m[:, d] = 1.0
        modes.append(m.ravel())
    for w in np.eye(3):
        modes.append(np.cross(w, X).ravel())
    for m in modes:
        assert np.linalg.norm(K @ m) <= 1e-11 * nK * np.linalg.norm(m)
    ev = np.linalg.eigvalsh(K)
    assert (np.abs(ev) < 1e-10 * ev.max()).sum() == 6
    assert ev[6] > 1e-7 * ev.max()


def test_uniform_tension_closed_form():
    E, nu, sig = 10000.0, 0.35, 3.0
    iso = dict(kind="iso", E=E, nu=nu)
    lam = block(3, 2, [(2, 1.0, 0, 0.0)], sx=4.0, sy=2.0, mats=[iso])
    lam.traction = [(1, (sig, 0.0, 0.0))]
    rollers = [inputs.clamp_face(lam, 0, (0,)), inputs.clamp_face(lam, 2, (1,)), inputs.clamp_face(lam, 4, (2,))]
    lam.dir_dof, lam.dir_val = inputs.merge_dirichlet(*rollers)
    mesh = fem.Mesh(lam)
    u = fem.System(mesh).direct().reshape(-1, 3)
    X = mesh.X
    exact = np.stack([sig * X[:, 0] / E, -nu * sig * X[:, 1] / E, -nu * sig * X[:, 2] / E], axis=1)
    assert np.abs(u - exact).max() <= 1e-11 * np.abs(exact).max()
    S = fem.element_stress_centre(mesh, u.ravel())
    assert np.allclose(S[:, 0, 0], sig, rtol=1e-10)
    assert np.abs(S[:, 1:, 1:]).max() < 1e-9 * sig


def test_pure_bending_exact_quadratic():
    """Pure bending of an isotropic beam: the 3D solution is quadratic, so Q2 is exact."""
    E, nu, kap = 10000.0, 0.3, 1e-3
    iso = dict(kind="iso", E=E, nu=nu)
    H, W, L = 1.5, 2.0, 6.0
    lam = block(4, 2, [(2, H, 0, 0.0)], sx=L, sy=np.array([-1.0, 0.2, 1.0]), mats=[iso])

    def exact(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2] - H / 2
        return np.stack([kap * x * z, -nu * kap * y * z, -0.5 * kap * (x * x + nu * (z * z - y * y))], axis=1)

    lam.traction = [(1, lambda x: (E * kap * (x[2] - H / 2), 0.0, 0.0))]
    mesh = fem.Mesh(lam)
    nodes = inputs.face_node_ids(lam, 0)
    dof = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    sysm = fem.System(mesh, dir_dof=dof, dir_val=exact(mesh.X[nodes]).ravel())
    u = sysm.direct()
    ex = exact(mesh.X).ravel()
    assert np.linalg.norm(u - ex) <= 1e-10 * np.linalg.norm(ex)


def test_tip_loaded_cantilever_approaches_timoshenko():
    """A clamped isotropic beam (L/h = 20) under a tip shear load: the 3D Q2
    solution approaches Timoshenko's P L^3/(3EI) + P L/(kGA), k = 5/6, within
    about 1% (the clamp's 3D constraint accounts for the rest) and settles
    under mesh refinement.  Convergence only, not an exact solution."""
    E, nu = 10000.0, 0.3
    G = E / (2 * (1 + nu))
    iso = dict(kind="iso", E=E, nu=nu)
    L, h, b, tau = 20.0, 1.0, 1.0, 0.01
    P, I, A = tau * b * h, b * h ** 3 / 12, b * h
    w_timo = P * L ** 3 / (3 * E * I) + P * L / (5 / 6 * G * A)
    tips = []
    for nx in (20, 40):
        lam = block(nx, 1, [(2, h, 0, 0.0)], sx=L, sy=b, mats=[iso])
        lam.traction = [(1, (0.0, 0.0, tau))]
        lam.dir_dof, lam.dir_val = inputs.clamp_face(lam, 0)
        mesh = fem.Mesh(lam)
        u = fem.System(mesh).direct().reshape(-1, 3)
        tips.append(u[np.isclose(mesh.X[:, 0], L), 2].mean())
    assert abs(tips[0] / w_timo - 1.0) <= 0.01 and abs(tips[1] / w_timo - 1.0) <= 0.01
    assert abs(tips[1] / tips[0] - 1.0) <= 0.005


def test_periodic_width_gives_generalised_plane_strain():
    """Periodic width conditions (the paper's 39-ply study, Section 3) on a
    homogeneous isotropic strip stretched along x: periodicity forbids a mean
    width strain, so the exact field is u = (eps x, 0, -nu/(1-nu) eps z), which
    Q2 reproduces; the same strip with free width faces contracts by -nu eps."""
    E, nu, eps, L, W, H = 10000.0, 0.3, 1e-3, 3.0, 2.0, 0.8
    iso = dict(kind="iso", E=E, nu=nu)
    lam = block(3, 2, [(2, H, 0, 0.0)], sx=L, sy=W, mats=[iso])
    mesh = fem.Mesh(lam)
    X = mesh.X
    ends = np.flatnonzero(np.isclose(X[:, 0], 0.0) | np.isclose(X[:, 0], L))
    corner = np.flatnonzero(np.all(np.isclose(X, 0.0), axis=1))
    above = np.flatnonzero(np.all(np.isclose(X, [0.0, 0.0, H]), axis=1))   # stops the rotation about x
    dof = np.concatenate([3 * ends, 3 * corner + 1, 3 * corner + 2, 3 * above + 1])
    val = np.concatenate([eps * X[ends, 0], [0.0], [0.0], [0.0]])
    u = fem.periodic_width_direct(mesh, dof, val, f=np.zeros(mesh.n_dof)).reshape(-1, 3)
    exact = np.stack([eps * X[:, 0], 0.0 * X[:, 0], -nu / (1 - nu) * eps * X[:, 2]], axis=1)
    assert np.abs(u - exact).max() <= 1e-12 * eps * L
    free = fem.System(mesh, f=np.zeros(mesh.n_dof), dir_dof=dof, dir_val=val).direct().reshape(-1, 3)
    assert np.allclose(free[:, 1], -nu * eps * X[:, 1], atol=1e-12)


def test_clt_laminate_in_plane_strain_exact():
    """[0/R/90/R/90/R/0] under in-plane strain: per-layer plane stress, reproduced exactly.

    u = (eps x, eps_y y, w(z)) with w' = -(C13 eps + C23 eps_y)/C33 per layer and
    eps_y from N_y = 0 of classical lamination theory (A = sum Qbar h).
    """
    c0 = inputs.flat_plate_c0()
    layers = list(zip([1] * 7, c0.layer_thick, c0.layer_mat, c0.layer_angle_deg))
    lam = block(2, 2, layers, sx=4.0, sy=4.0)
    Cply = fem.orthotropic_C(**inputs.PLY_T1)
    perm = [1, 0, 2, 4, 3, 5]
    Cl = {0.0: Cply, 90.0: Cply[np.ix_(perm, perm)]}
    Ciso = fem.isotropic_C(**inputs.RESIN_T1)
    Cs = [Ciso if m == 1 else Cl[a] for m, a in zip(lam.layer_mat, lam.layer_angle_deg)]
    Qb = [C[:2, :2] - np.outer(C[:2, 2], C[2, :2]) / C[2, 2] for C in Cs]
    A = sum(Q * h for Q, h in zip(Qb, lam.layer_thick))
    eps = 1e-3
    eps_y = -A[1, 0] / A[1, 1] * eps
    ez = [-(C[0, 2] * eps + C[1, 2] * eps_y) / C[2, 2] for C in Cs]
    zb = np.concatenate([[0.0], np.cumsum(lam.layer_thick)])

    def w(z):
        k = np.clip(np.searchsorted(zb, z, side="right") - 1, 0, len(ez) - 1)
        return np.array([sum(ez[i] * lam.layer_thick[i] for i in range(kk)) + ez[kk] * (zz - zb[kk])
                         for kk, zz in zip(k, z)])

    mesh = fem.Mesh(lam)
    sides = np.unique(np.concatenate([inputs.face_node_ids(lam, f) for f in (0, 1, 2, 3)]))
    bottom = inputs.face_node_ids(lam, 4)
    X = mesh.X
    dof = np.concatenate([3 * sides, 3 * sides + 1, 3 * bottom + 2])
    val = np.concatenate([eps * X[sides, 0], eps_y * X[sides, 1], np.zeros(bottom.size)])
    dof, val = inputs.merge_dirichlet((dof, val))
    u = fem.System(mesh, f=np.zeros(mesh.n_dof), dir_dof=dof, dir_val=val).direct().reshape(-1, 3)
    ex = np.stack([eps * X[:, 0], eps_y * X[:, 1], w(X[:, 2])], axis=1)
    assert np.abs(u - ex).max() <= 1e-10 * np.abs(ex).max()
    S = fem.element_stress_centre(mesh, u.ravel())
    s33, t13 = fem.stress_slr(mesh, u.ravel())
    lay = mesh.layer_of_elem
    sx_exact = np.array([Qb[k][0, 0] * eps + Qb[k][0, 1] * eps_y for k in lay])
    assert np.allclose(S[:, 0, 0], sx_exact, rtol=1e-8)
    assert np.abs(s33).max() < 1e-8 * np.abs(sx_exact).max()
    assert np.abs(t13).max() < 1e-8 * np.abs(sx_exact).max()


def test_free_edge_plate_modulus_near_clt():
    """The [0/R/90/R/90/R/0] plate stretched along x with free width and thickness
    faces: its axial stiffness F/(eps W) is the CLT membrane stiffness
    A11 - A12^2/A22 up to free-edge effects of about a percent."""
    c0 = inputs.flat_plate_c0()
    layers = list(zip([1] * 7, c0.layer_thick, c0.layer_mat, c0.layer_angle_deg))
    L = W = 20.0
    lam = block(8, 8, layers, sx=L, sy=W)
    Cply = fem.orthotropic_C(**inputs.PLY_T1)
    perm = [1, 0, 2, 4, 3, 5]
    Cl = {0.0: Cply, 90.0: Cply[np.ix_(perm, perm)]}
    Ciso = fem.isotropic_C(**inputs.RESIN_T1)
    Cs = [Ciso if m == 1 else Cl[a] for m, a in zip(lam.layer_mat, lam.layer_angle_deg)]
    Qb = [C[:2, :2] - np.outer(C[:2, 2], C[2, :2]) / C[2, 2] for C in Cs]
    A = sum(Q * h for Q, h in zip(Qb, lam.layer_thick))
    a_clt = A[0, 0] - A[0, 1] ** 2 / A[1, 1]
    mesh = fem.Mesh(lam)
    X = mesh.X
    eps = 1e-3
    ends = np.flatnonzero(np.isclose(X[:, 0], 0.0) | np.isclose(X[:, 0], L))
    o = np.flatnonzero(np.all(np.isclose(X, 0.0), axis=1))
    oy = np.flatnonzero(np.all(np.isclose(X, [0.0, W, 0.0]), axis=1))
    dof = np.concatenate([3 * ends, 3 * o + 1, 3 * o + 2, 3 * oy + 2])
    val = np.concatenate([eps * X[ends, 0], [0.0, 0.0, 0.0]])
    sysm = fem.System(mesh, f=np.zeros(mesh.n_dof), dir_dof=dof, dir_val=val)
    u = sysm.direct()
    far = np.flatnonzero(np.isclose(X[:, 0], L))
    F = (sysm.K @ u)[3 * far].sum()
    assert abs(F / (eps * W) / a_clt - 1.0) <= 0.03


def test_rigid_rotation_gives_zero_stress_on_curved_mesh():
    lam = inputs.corner_mini(n_arc=4, n_limb=1, n_width=2, nel_layer=1)
    mesh = fem.Mesh(lam)
    w = np.array([2e-3, -1e-3, 3e-3])
    u = (np.cross(w, mesh.X) + np.array([1e-3, 2e-3, 0.0])).ravel()
    s33, t13 = fem.stress_slr(mesh, u)
    assert max(np.abs(s33).max(), np.abs(t13).max()) < 1e-9 * 162000.0 * 3e-3


def test_curved_map_geometry():
    lam = inputs.corner_mini(n_arc=6, n_limb=2, n_width=2, nel_layer=1)
    mesh = fem.Mesh(lam)
    t = fem.q2_node_params(lam.sv)
    on_arc = (t >= 0) & (t <= 1)
    X = mesh.X.reshape(mesh.NZ, mesh.NY, mesh.NX, 3)
    rn = lam.R_inner + fem.q2_node_params(fem.rv_vertices(lam))
    rad = np.hypot(X[:, :, on_arc, 0] - lam.limb_L, X[:, :, on_arc, 2])
    assert np.allclose(rad, rn[:, None, None] * np.ones_like(rad), rtol=1e-14)
    # limb 1 is horizontal at height r, limb 2 vertical at x = L + r
    assert np.allclose(X[:, :, 0, 2], rn[:, None])
    assert np.allclose(X[:, :, -1, 0], lam.limb_L + rn[:, None])


# --------------------------------------------------------------------------- orientation conventions
#
# The material axes and the stress frame are fixed by the geometry: a fibre
# runs along the ply (the tangent of the mapped mesh), a ply angle turns it
# about the outward normal r from s toward the width axis l (the usual
# laminate convention; the paper gives stacks such as [0/90/+45/-45]s without
# fixing the sign, Section 2.2), and sigma_33 is the normal stress on the
# through-thickness direction of the curved laminate (Section 2.2 notation,
# Section 3 map).  These pins measure the stiffest direction of C_e and the
# frame from node positions, not from the oracle's rotation matrices.


def _stiffness_along(C, n):
    """Directional stiffness e^T C e of the uniaxial strain n (x) n (Voigt, engineering shears), rows of n."""
    n = np.atleast_2d(n)
    e = np.stack([n[:, 0] ** 2, n[:, 1] ** 2, n[:, 2] ** 2, 2 * n[:, 1] * n[:, 2], 2 * n[:, 0] * n[:, 2],
                  2 * n[:, 0] * n[:, 1]], axis=1)
    return np.einsum("ni,ij,nj->n", e, C, e)


def _stiffest_direction(C):
    """Unit n maximising the quartic e(n)^T C e(n): best of 20,000 Fibonacci-sphere
    samples, refined by the shifted symmetric higher-order power method
    (n <- normalise(grad/4 + a n), monotone for a shift a above the quartic's
    curvature bound)."""
    k = np.arange(20000) + 0.5
    z = 1.0 - 2.0 * k / k.size
    rho = np.sqrt(1.0 - z * z)
    ph = math.pi * (1.0 + math.sqrt(5.0)) * k
    pts = np.stack([rho * np.cos(ph), rho * np.sin(ph), z], axis=1)
    n = pts[np.argmax(_stiffness_along(C, pts))]
    a = 4.0 * np.abs(C).sum()
    for _ in range(5000):
        e = np.array([n[0] ** 2, n[1] ** 2, n[2] ** 2, 2 * n[1] * n[2], 2 * n[0] * n[2], 2 * n[0] * n[1]])
        D = np.array([[2 * n[0], 0, 0], [0, 2 * n[1], 0], [0, 0, 2 * n[2]], [0, 2 * n[2], 2 * n[1]],
                      [2 * n[2], 0, 2 * n[0]], [2 * n[1], 2 * n[0], 0]])
        g = 2.0 * D.T @ (C @ e)
        m = g / 4.0 + a * n
        m /= np.linalg.norm(m)
        if np.linalg.norm(m - n) < 1e-15:
            n = m
            break
        n = m
    return n


def _angle(a, b):
    c = abs(float(np.dot(a, b))) / (np.linalg.norm(a) * np.linalg.norm(b))
    return math.acos(min(1.0, c))


def test_fibre_follows_the_arc_tangent_and_ply_angle():
    """On a curved corner without misalignment, the stiffest direction of every
    ply element's C_e is cos(phi) t + sin(phi) e_l, with t the unit tangent of
    the mapped mesh at the element centre taken from two node positions (the
    chord between the centres of the element's -s and +s faces, parallel to
    the arc's tangent at the centre and exact on the limbs)."""
    lam = inputs.corner_mini(n_arc=6, n_limb=1, n_width=2, nel_layer=1, angles=(0, 45, -45, 90), amp_deg=0.0)
    mesh = fem.Mesh(lam)
    assert np.all(mesh.theta == 0.0)
    phi = np.radians(np.asarray(lam.layer_angle_deg, dtype=np.float64))[mesh.layer_of_elem]
    psi_seen = set()
    checked = 0
    for e in range(0, mesh.n_elem, 3):
        if mesh.is_resin[e]:
            continue
        t = mesh.X[mesh.conn[e][14]] - mesh.X[mesh.conn[e][12]]
        t /= np.linalg.norm(t)
        fibre = math.cos(phi[e]) * t + math.sin(phi[e]) * np.array([0.0, 1.0, 0.0])
        n = _stiffest_direction(mesh.C[e])
        assert _angle(n, fibre) <= 1e-6, (e, n, fibre)
        psi_seen.add(round(float(mesh.psi[e]), 6))
        checked += 1
    assert checked > 20 and len(psi_seen) >= 5       # limbs and several arc positions


def test_positive_ply_angle_turns_the_fibre_toward_the_width_axis():
    """Flat plate: a +45 ply is stiffest along (1, 1, 0)/sqrt 2, a -45 ply along
    (1, -1, 0)/sqrt 2, a 90 ply along the width axis, a 0 ply along s."""
    lam = block(1, 1, [(1, 0.25, 0, 45.0), (1, 0.25, 0, -45.0), (1, 0.25, 0, 90.0), (1, 0.25, 0, 0.0)])
    mesh = fem.Mesh(lam)
    r2 = 1.0 / math.sqrt(2.0)
    want = [np.array([r2, r2, 0.0]), np.array([r2, -r2, 0.0]), np.array([0.0, 1.0, 0.0]),
            np.array([1.0, 0.0, 0.0])]
    for e, w in enumerate(want):
        assert _angle(_stiffest_direction(mesh.C[e]), w) <= 1e-6
    # misalignment tilts a 0 ply's fibre in the s-r plane: theta > 0 turns it from +s toward -r
    lam.theta = np.full((4, 1, 1), 0.2)
    mesh = fem.Mesh(lam)
    n = _stiffest_direction(mesh.C[3])
    assert _angle(n, np.array([math.cos(0.2), 0.0, -math.sin(0.2)])) <= 1e-6


def test_curved_stress_frame_from_positions():
    """Homogeneous isotropic corner under a linear displacement u = A x: the
    stress is the same tensor S everywhere (Q2 holds linear fields exactly),
    and sigma_33, tau_13 returned per element must equal n_r^T S n_r and
    n_s^T S n_r with n_r the outward radial unit vector computed from the
    element centre's position (x_c - L, 0, z_c) on the arc, (0, 0, 1) on limb 1
    and (1, 0, 0) on limb 2 of the 90-degree corner, and n_s = n_l x n_r the
    direction of increasing s."""
    lam = inputs.corner_mini(n_arc=6, n_limb=1, n_width=2, nel_layer=1, angles=(0, 90), amp_deg=0.0)
    lam.layer_mat = [1] * len(lam.layer_mat)            # resin everywhere: C uniform
    mesh = fem.Mesh(lam)
    rng = np.random.default_rng(7)
    A = rng.standard_normal((3, 3)) * 1e-3
    u = (mesh.X @ A.T).ravel()
    E, nu = inputs.RESIN_T1["E"], inputs.RESIN_T1["nu"]
    eps = 0.5 * (A + A.T)
    S = E / (1 + nu) * (eps + nu / (1 - 2 * nu) * np.trace(eps) * np.eye(3))
    s33, t13 = fem.stress_slr(mesh, u)
    t = fem.q2_node_params(lam.sv)
    for e in range(mesh.n_elem):
        xc = mesh.X[mesh.conn[e][13]]
        ex = mesh.eijk[e, 0]
        tc = t[2 * ex + 1]
        if tc < 0.0:
            nr = np.array([0.0, 0.0, 1.0])
        elif tc > 1.0:
            nr = np.array([1.0, 0.0, 0.0])
        else:
            nr = np.array([xc[0] - lam.limb_L, 0.0, xc[2]])
            nr /= np.linalg.norm(nr)
        ns = np.cross(np.array([0.0, 1.0, 0.0]), nr)
        assert abs(s33[e] - nr @ S @ nr) <= 1e-10 * np.abs(S).max()
        assert abs(t13[e] - ns @ S @ nr) <= 1e-10 * np.abs(S).max()
    assert np.ptp(s33) > 0.1 * np.abs(S).max()         # the frame really turns


def test_direct_solvers_agree_with_dense_cholesky():
    lam = inputs.corner_mini(n_arc=3, n_limb=1, n_width=2, nel_layer=1, nsub=(2, 1, 1), nev=6)
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    A = sysm.Kff.toarray()
    L = np.linalg.cholesky(A)
    x_dense = np.linalg.solve(L.T, np.linalg.solve(L, sysm.ff))
    u = sysm.direct()
    assert np.linalg.norm(u[sysm.free] - x_dense) <= 1e-10 * np.linalg.norm(x_dense)
    u2, it, hist, P, _ = geneo.solve(lam, system=sysm, tol=1e-13)
    assert hist[-1] <= 1e-13
    assert np.linalg.norm(u2 - u) <= 1e-9 * np.linalg.norm(u)


# --------------------------------------------------------------------------- GenEO


@pytest.fixture(scope="module")
def small_geneo():
    lam = inputs.corner_mini(n_arc=4, n_limb=1, n_width=4, nel_layer=1, nsub=(3, 2, 1), nev=8)
    sysm = fem.System(fem.Mesh(lam))
    dec = geneo.Decomposition(sysm, 3, 2, 1, 1)
    return lam, sysm, dec, geneo.GenEO(dec, 8)


def test_partition_of_unity(small_geneo):
    lam, sysm, dec, P = small_geneo
    acc = np.zeros(sysm.free.size)
    for s in dec.subs:
        acc[s.VN] += s.xi
    assert np.abs(acc - 1.0).max() < 1e-14


def test_preconditioner_symmetric_positive(small_geneo):
    lam, sysm, dec, P = small_geneo
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((2, sysm.free.size))
    a, b = x @ P.apply(y), y @ P.apply(x)
    assert abs(a - b) <= 1e-12 * max(abs(a), 1e-30) * 10
    assert x @ P.apply(x) > 0


def test_floating_subdomain_rigid_modes_in_coarse_space(small_geneo):
    lam, sysm, dec, P = small_geneo
    X = sysm.mesh.X
    free = sysm.free
    floating = 0
    for j, s in enumerate(dec.subs):
        touches_clamp = s.box[0][0] == 0 or s.box[0][1] == lam.nx   # both limb ends are Dirichlet
        lamv = P.eigvals[j]
        n0 = int((np.abs(lamv) < 1e-9).sum())
        assert n0 == (0 if touches_clamp else 6)
        if touches_clamp:
            continue
        floating += 1
        Zj = P.Z[:, j * 8:(j + 1) * 8].toarray()[s.VN]
        for w in np.eye(3):
            rig = np.cross(w, X).ravel()[free][s.VN] * s.xi
            coef, *_ = np.linalg.lstsq(Zj, rig, rcond=None)
            assert np.linalg.norm(Zj @ coef - rig) <= 1e-8 * np.linalg.norm(rig)
    assert floating >= 1


def test_geneo_dense_vs_arpack_and_shift_independence(small_geneo):
    lam, sysm, dec, P = small_geneo
    s = dec.subs[1]
    AN = dec.neumann_matrix(s)
    l1, _ = geneo.geneo_eigs(AN, s.xi, 8, method="dense")
    l2, _ = geneo.geneo_eigs(AN, s.xi, 8, method="arpack")
    l3, _ = geneo.geneo_eigs(AN, s.xi, 8, method="dense", sigma=0.3)
    assert np.allclose(l1, l2, rtol=1e-7, atol=1e-9)
    assert np.allclose(l1, l3, rtol=1e-7, atol=1e-9)


def _strip(ns):
    nel, th, mat, ang = inputs._stack_with_resin([0, 90, 0], 0.25, 0.02, 1, 1)
    lam = inputs.Laminate(name="strip", geometry=0, sv=np.linspace(0, 3 * ns, 3 * ns + 1),
                          lv=np.linspace(0, 2.0, 3), layer_nel=nel, layer_thick=th, layer_mat=mat,
                          layer_angle_deg=ang, materials=[inputs.PLY_T1, inputs.RESIN_T1])
    lam.dir_dof, lam.dir_val = inputs.clamp_face(lam, 0)
    lam.traction = [(1, (0.0, 0.0, 1.0))]
    return lam


def test_independent_columns_match_rank():
    """Dependent-column dropping keeps a basis of the column space: a duplicated
    column, a linear combination and a zero column go; the count equals the
    rank from numpy's SVD and the kept Gram block is positive definite."""
    rng = np.random.default_rng(8)
    G = rng.standard_normal((60, 12))
    G[:, 5] = G[:, 1]
    G[:, 8] = 2.0 * G[:, 0] - 3.0 * G[:, 3]
    G[:, 10] = 0.0
    K0 = G.T @ G
    keep = geneo.independent_columns(K0)
    assert list(keep) == [j for j in range(12) if j not in (5, 8, 10)]
    assert len(keep) == np.linalg.matrix_rank(G)
    np.linalg.cholesky(K0[np.ix_(keep, keep)])


def test_coincident_subdomains_drop_coarse_columns():
    """A laminate two elements wide split in two across its width with overlap 1:
    both subdomains of each pair grow to the full width and coincide, so half
    of their GenEO vectors are dependent.  The dropped columns lie in the span
    of the kept ones (the K-orthogonal coarse projector reproduces them) and
    PCG still converges to the direct solution."""
    lam = inputs.corner_mini(n_arc=4, n_limb=1, n_width=2, nel_layer=1, angles=(0, 90), nsub=(2, 2, 1), nev=6,
                             limb_L=2.0, width=2.0)
    sysm = fem.System(fem.Mesh(lam))
    dec = geneo.Decomposition(sysm, 2, 2, 1, 1)
    sets = [tuple(np.sort(s.VN)) for s in dec.subs]
    pairs = sum(1 for i in range(len(sets)) for j in range(i) if sets[i] == sets[j])
    assert pairs == 2
    P = geneo.GenEO(dec, 6, eig_method="dense")
    assert P.n_dropped == 6 * pairs
    K = sysm.Kff
    Z, Za = P.Z.toarray(), P.Z_all.toarray()
    proj = Z @ sla_solve(P.K0, Z.T @ (K @ Za))
    assert np.abs(proj - Za).max() <= 1e-8 * np.abs(Za).max()
    u, it, hist, _, _ = geneo.solve(lam, system=sysm, px=2, py=2, pz=1, nev=6, tol=1e-12)
    ud = sysm.direct()
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)


def test_geneo_iterations_flat_while_one_level_grows():
    """Section 2.3: GenEO iterations stay roughly constant as subdomains are added,
    one-level Schwarz iterations grow (the paper reports ~40 against ~400)."""
    its, its1 = [], []
    for ns in (4, 16):
        lam = _strip(ns)
        sysm = fem.System(fem.Mesh(lam))
        dec = geneo.Decomposition(sysm, ns, 1, 1, 1)
        _, it, _ = geneo.pcg(sysm.Kff, sysm.ff, geneo.GenEO(dec, 8).apply, tol=1e-10)
        _, it1, _ = geneo.pcg(sysm.Kff, sysm.ff, geneo.GenEO(dec, 8, coarse=False).apply, tol=1e-10)
        its.append(it)
        its1.append(it1)
    assert its[1] <= 1.6 * its[0]
    assert its1[1] >= 4 * its1[0]
    assert its[1] * 3 < its1[1]


# --------------------------------------------------------------------------- adjoint


def test_oracle_adjoint_gradient_matches_central_differences():
    """The oracle's adjoint dJ/dtheta of J = ||s33||_8 over the arc resin elements
    agrees with central differences of J (direct solves, h = 1e-6 rad)."""
    from oracle import adjoint
    lam = inputs.corner_mini(n_arc=4, n_limb=1, n_width=2, nel_layer=1, angles=(0, 90), limb_L=2.0, width=2.0)
    mesh = fem.Mesh(lam)
    tc = 0.5 * (lam.sv[mesh.eijk[:, 0]] + lam.sv[mesh.eijk[:, 0] + 1])
    mask = mesh.is_resin & (tc > 0) & (tc < 1)
    J, grad, u = adjoint.gradient(fem.System(mesh), mask, 8)
    assert J > 0
    theta0 = mesh.theta.copy()
    plies = np.nonzero(~mesh.is_resin)[0]
    picks = plies[np.argsort(-np.abs(grad[plies]))[:3]]
    h = 1e-6
    for e in picks:
        tp, tm = theta0.copy(), theta0.copy()
        tp[e] += h
        tm[e] -= h
        fd = (adjoint.objective_at(lam, tp, mask, 8) - adjoint.objective_at(lam, tm, mask, 8)) / (2 * h)
        assert abs(fd - grad[e]) <= 1e-6 * np.abs(grad).max()
    assert np.all(grad[mesh.is_resin & ~mask] == 0.0)


def test_oracle_adjoint_step_sweep_shows_second_order_differences():
    """Central differences of J against the oracle's adjoint gradient over
    h = 1e-2 .. 1e-6 rad: the error falls as h^2 (a factor ~100 per decade)
    until rounding takes over, where it stays below 1e-6 relative."""
    from oracle import adjoint
    lam = inputs.corner_mini(n_arc=4, n_limb=1, n_width=2, nel_layer=1, angles=(0, 90), limb_L=2.0, width=2.0)
    mesh = fem.Mesh(lam)
    mask = inputs.arc_resin_mask(lam)
    J, grad, u = adjoint.gradient(fem.System(mesh), mask, 8)
    theta0 = mesh.theta.copy()
    plies = np.nonzero(~mesh.is_resin)[0]
    e = plies[np.argmax(np.abs(grad[plies]))]
    err = []
    for h in (1e-2, 1e-3, 1e-4, 1e-6):
        tp, tm = theta0.copy(), theta0.copy()
        tp[e] += h
        tm[e] -= h
        fd = (adjoint.objective_at(lam, tp, mask, 8) - adjoint.objective_at(lam, tm, mask, 8)) / (2 * h)
        err.append(abs(fd - grad[e]) / abs(grad[e]))
    assert 70.0 <= err[0] / err[1] <= 130.0
    assert err[1] / err[2] >= 40.0
    assert err[3] <= 1e-6


def test_failure_index_uniform_stress_closed_form():
    """Eq. eq-Camanho on a resin block under a uniform strain: sigma = C eps is known
    in closed form, so F = sqrt((max(s_zz,0)/61)^2 + (s_xz/97)^2 + (s_yz/97)^2)."""
    iso = dict(kind="iso", E=10000.0, nu=0.35)
    lam = block(2, 2, [(2, 1.0, 0, 0.0)], sx=2.0, sy=2.0, mats=[iso])
    mesh = fem.Mesh(lam)
    for sign in (1.0, -1.0):
        eps = np.array([[1e-4, 2e-4, 3e-4], [2e-4, -1e-4, 5e-4], [3e-4, 5e-4, sign * 4e-4]])
        u = (mesh.X @ eps.T).ravel()
        Cv = fem.isotropic_C(**iso)
        ev = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[1, 2], 2 * eps[0, 2], 2 * eps[0, 1]])
        s = Cv @ ev
        F_exact = np.sqrt((max(s[2], 0.0) / 61.0) ** 2 + (s[4] / 97.0) ** 2 + (s[3] / 97.0) ** 2)
        F = fem.failure_index(mesh, u)
        assert np.allclose(F, F_exact, rtol=1e-12)

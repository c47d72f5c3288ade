"""Pins for the oracle's 20-node serendipity element (no GPU): the element the
paper's own code uses, kept as the oracle of a future GPU version."""
import numpy as np

from oracle import fem, serendipity
from paper_1707_04228_gb300 import inputs


def block(nx, ny, layers, sx=1.0, sy=1.0, mats=None, geometry=0, **kw):
    nel, th, mat, ang = (list(t) for t in zip(*layers))
    sv = np.linspace(0.0, sx, nx + 1) if np.isscalar(sx) else np.asarray(sx)
    lv = np.linspace(0.0, sy, ny + 1) if np.isscalar(sy) else np.asarray(sy)
    return inputs.Laminate(name="t", geometry=geometry, sv=sv, lv=lv, layer_nel=nel, layer_thick=th,
                           layer_mat=mat, layer_angle_deg=ang, materials=mats or [inputs.PLY_T1, inputs.RESIN_T1],
                           **kw)


def test_shape_functions_kronecker_unity_and_gradients():
    ref = serendipity._REF
    for b, r in enumerate(ref):
        N, _ = serendipity.shape20(*r)
        assert np.allclose(N, np.eye(20)[b], atol=1e-14)
    rng = np.random.default_rng(0)
    h = 1e-6
    for p in rng.uniform(-1, 1, (5, 3)):
        N, dN = serendipity.shape20(*p)
        assert abs(N.sum() - 1.0) < 1e-14 and np.abs(dN.sum(axis=0)).max() < 1e-13
        # every gradient against central differences of the shape functions themselves
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fd = (serendipity.shape20(*(p + e))[0] - serendipity.shape20(*(p - e))[0]) / (2 * h)
            assert np.abs(fd - dN[:, d]).max() < 1e-8
        # quadratic monomials are reproduced: sum_a N_a q(x_a) = q(x)
        for q in (lambda x: x[0] * x[1], lambda x: x[2] ** 2, lambda x: x[0] * x[2] + x[1] ** 2):
            assert abs(N @ np.array([q(r) for r in ref]) - q(p)) < 1e-14


def test_node_count_of_the_plate():
    """Vertices plus edge midpoints of the 8x8x14 plate: 9*9*15 + 8*9*15 + 9*8*15 + 9*9*14
    = 4,509 nodes, 13,527 DOF."""
    m = serendipity.Mesh20(inputs.flat_plate_c0())
    assert m.n_nodes == 9 * 9 * 15 + 8 * 9 * 15 + 9 * 8 * 15 + 9 * 9 * 14
    assert m.n_dof == 13_527


def _boundary(mesh):
    X = mesh.X
    lo, hi = X.min(axis=0), X.max(axis=0)
    return np.flatnonzero(np.any(np.isclose(X, lo) | np.isclose(X, hi), axis=1))


def _solve_linear_patch(lam, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((3, 3)) * 1e-3
    b = rng.standard_normal(3) * 1e-3
    m = serendipity.Mesh20(lam)
    K = m.assemble_K()
    if lam.geometry == 0:
        nodes = _boundary(m)
    else:   # boundary of the parametric box: nodes on the first/last grid plane of any axis
        q2 = m.q2
        n = m.q2_of
        ix, iy, iz = n % q2.NX, (n // q2.NX) % q2.NY, n // (q2.NX * q2.NY)
        nodes = np.flatnonzero((ix == 0) | (ix == q2.NX - 1) | (iy == 0) | (iy == q2.NY - 1) | (iz == 0)
                               | (iz == q2.NZ - 1))
    dof = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    u = serendipity.solve_dirichlet(m, K, np.zeros(m.n_dof), dof, (m.X[nodes] @ A.T + b).ravel())
    exact = (m.X @ A.T + b).ravel()
    return np.linalg.norm(u - exact) / np.linalg.norm(exact)


def test_patch_test_flat_and_curved():
    iso = dict(kind="iso", E=10000.0, nu=0.3)
    flat = block(3, 2, [(2, 0.6, 0, 30.0)], sx=[0.0, 0.4, 1.5, 2.0], sy=[0.0, 0.8, 1.1])
    assert _solve_linear_patch(flat, 1) <= 1e-11
    curved = block(4, 2, [(2, 0.4, 0, 0.0)], sx=inputs.graded(4, -1.0, 2.0, 3.0), sy=[0.0, 0.7, 2.0],
                   mats=[iso], geometry=1, R_inner=2.0, limb_L=1.5, arc_deg=90.0)
    assert _solve_linear_patch(curved, 2) <= 1e-11


def test_pure_bending_is_exact():
    """The pure-bending field is quadratic, inside the serendipity space on box elements."""
    E, nu, kap, H = 10000.0, 0.3, 1e-3, 1.5
    lam = block(4, 2, [(2, H, 0, 0.0)], sx=6.0, sy=np.array([-1.0, 0.2, 1.0]), mats=[dict(kind="iso", E=E, nu=nu)])

    def exact(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2] - H / 2
        return np.stack([kap * x * z, -nu * kap * y * z, -0.5 * kap * (x * x + nu * (z * z - y * y))], axis=1)

    m = serendipity.Mesh20(lam)
    K = m.assemble_K()
    nodes = _boundary(m)
    dof = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    u = serendipity.solve_dirichlet(m, K, np.zeros(m.n_dof), dof, exact(m.X[nodes]).ravel())
    ex = exact(m.X).ravel()
    assert np.linalg.norm(u - ex) <= 1e-10 * np.linalg.norm(ex)


def test_six_rigid_body_modes_on_a_free_body():
    lam = block(2, 1, [(1, 0.4, 0, 45.0), (1, 0.1, 1, 0.0)], sx=1.5, sy=1.0)
    K = serendipity.Mesh20(lam).assemble_K().toarray()
    w = np.linalg.eigvalsh(K)
    assert np.all(np.abs(w[:6]) <= 1e-10 * w[-1]) and w[6] > 1e-6 * w[-1]


def test_matches_q2_on_a_converged_cantilever():
    """Both elements converge to the same tip deflection of a clamped beam under a
    tip shear load (L/h = 20), within 0.5%."""
    E, nu = 10000.0, 0.3
    iso = dict(kind="iso", E=E, nu=nu)
    lam = block(20, 1, [(2, 1.0, 0, 0.0)], sx=20.0, sy=1.0, mats=[iso])
    lam.traction = [(1, (0.0, 0.0, 0.01))]
    lam.dir_dof, lam.dir_val = inputs.clamp_face(lam, 0)
    q2 = fem.Mesh(lam)
    f_q2 = fem.load_vector(q2)
    u_q2 = fem.System(q2).direct().reshape(-1, 3)
    w_q2 = u_q2[np.isclose(q2.X[:, 0], 20.0), 2].mean()
    m = serendipity.Mesh20(lam)
    K = m.assemble_K()
    # consistent load of a uniform traction on the face x = L: its resultant split by the
    # serendipity face weights (corners -1/12, edge midpoints 1/3 of the face-area share)
    f = np.zeros(m.n_dof)
    tip = np.flatnonzero(np.isclose(m.X[:, 0], 20.0))
    face_elems = np.flatnonzero(np.isclose(m.X[m.conn][:, :, 0].max(axis=1), 20.0))
    gq, wq = fem.gauss3()
    for e in face_elems:
        Xe = m.X[m.conn[e]]
        for i, a in enumerate(gq):
            for j, b in enumerate(gq):
                N, dN = serendipity.shape20(1.0, a, b)
                J = Xe.T @ dN
                dA = np.linalg.norm(np.cross(J[:, 1], J[:, 2]))
                f[3 * m.conn[e] + 2] += wq[i] * wq[j] * dA * 0.01 * N
    assert abs(f.sum() - 0.01 * 1.0 * 1.0) < 1e-12 and abs(f.sum() - f_q2.sum()) < 1e-12
    clamp = np.flatnonzero(np.isclose(m.X[:, 0], 0.0))
    dof = (3 * clamp[:, None] + np.arange(3)[None, :]).ravel()
    u = serendipity.solve_dirichlet(m, K, f, dof, np.zeros(dof.size)).reshape(-1, 3)
    w20 = u[tip, 2].mean()
    assert abs(w20 / w_q2 - 1.0) <= 0.005


def test_uniform_traction_closed_form_nodal_shares():
    """The 8-node serendipity face loaded by a uniform traction on a rectangle
    of area A: each corner node receives -A t / 12 and each mid-side node
    A t / 3 (the textbook consistent loads of the quadratic serendipity
    quadrilateral); summed over the elements of a face, every node gets the
    sum of its shares, and the total is the face area times t."""
    lam = block(3, 2, [(2, 0.5, 1, 0.0)], sx=[0.0, 1.0, 2.5, 3.0], sy=[0.0, 0.8, 2.0])
    m = serendipity.Mesh20(lam)
    t = np.array([1.0, -2.0, 0.5])
    f = serendipity.traction_load20(m, 1, t).reshape(-1, 3)   # face +s at x = 3
    expect = np.zeros_like(f)
    ly = lam.lv
    z = np.cumsum([0.0] + [0.5 / 2] * 2)
    for iy in range(len(ly) - 1):
        for iz in range(2):
            A = (ly[iy + 1] - ly[iy]) * (z[iz + 1] - z[iz])
            corners = [(ly[iy], z[iz]), (ly[iy + 1], z[iz]), (ly[iy], z[iz + 1]), (ly[iy + 1], z[iz + 1])]
            mids = [(0.5 * (ly[iy] + ly[iy + 1]), z[iz]), (0.5 * (ly[iy] + ly[iy + 1]), z[iz + 1]),
                    (ly[iy], 0.5 * (z[iz] + z[iz + 1])), (ly[iy + 1], 0.5 * (z[iz] + z[iz + 1]))]
            for pts, share in ((corners, -A / 12.0), (mids, A / 3.0)):
                for (y, zz) in pts:
                    k = np.flatnonzero(np.isclose(m.X[:, 0], 3.0) & np.isclose(m.X[:, 1], y) & np.isclose(m.X[:, 2], zz))
                    assert k.size == 1
                    expect[k[0]] += share * t
    assert np.abs(f - expect).max() <= 1e-13
    assert np.allclose(f.sum(axis=0), 2.0 * 0.5 * t, rtol=1e-14)


def test_uniform_tension_with_traction_loads_is_exact():
    """Isotropic bar with roller supports on x = 0, y = 0, z = 0 and a uniform
    x-traction s on x = L: the solution u = (s x / E, -nu s y / E, -nu s z / E)
    is linear, so the serendipity element reproduces it to round-off."""
    lam = block(4, 2, [(3, 0.9, 1, 0.0)], sx=[0.0, 0.5, 1.5, 2.2, 3.0], sy=[0.0, 0.7, 1.2])
    m = serendipity.Mesh20(lam)
    E, nu, s = inputs.RESIN_T1["E"], inputs.RESIN_T1["nu"], 5.0
    K = m.assemble_K()
    f = serendipity.traction_load20(m, 1, (s, 0.0, 0.0))
    X = m.X
    dof = np.concatenate([3 * np.flatnonzero(np.isclose(X[:, 0], 0.0)),
                          3 * np.flatnonzero(np.isclose(X[:, 1], 0.0)) + 1,
                          3 * np.flatnonzero(np.isclose(X[:, 2], 0.0)) + 2])
    u = serendipity.solve_dirichlet(m, K, f, dof, np.zeros(dof.size))
    exact = np.stack([s * X[:, 0] / E, -nu * s * X[:, 1] / E, -nu * s * X[:, 2] / E], axis=1).ravel()
    assert np.linalg.norm(u - exact) <= 1e-10 * np.linalg.norm(exact)


def test_centre_stress_uniform_tension_and_rigid_rotation():
    """Uniform tension: every centre stress is sigma_xx = s (sigma_33 = tau_13 = 0
    on the flat bar); a rigid rotation of a curved serendipity corner gives zero
    stress (the frame and the 20-node map agree)."""
    lam = block(4, 2, [(3, 0.9, 1, 0.0)], sx=[0.0, 0.5, 1.5, 2.2, 3.0], sy=[0.0, 0.7, 1.2])
    m = serendipity.Mesh20(lam)
    E, nu, s = inputs.RESIN_T1["E"], inputs.RESIN_T1["nu"], 5.0
    X = m.X
    u = np.stack([s * X[:, 0] / E, -nu * s * X[:, 1] / E, -nu * s * X[:, 2] / E], axis=1).ravel()
    s33, t13 = serendipity.stress_slr20(m, u)
    assert np.abs(s33).max() < 1e-12 * s and np.abs(t13).max() < 1e-12 * s
    # the rotated frame sees the axial stress on a tilted plane: check sigma_xx via a 90-degree corner limb
    lamc = inputs.corner_mini(n_arc=4, n_limb=1, n_width=2, nel_layer=1)
    mc = serendipity.Mesh20(lamc)
    w = np.array([2e-3, -1e-3, 3e-3])
    uc = (np.cross(w, mc.X) + np.array([1e-3, 2e-3, 0.0])).ravel()
    c33, c13 = serendipity.stress_slr20(mc, uc)
    assert max(np.abs(c33).max(), np.abs(c13).max()) < 1e-9 * 162000.0 * 3e-3


def test_centre_stress_of_a_field_in_both_spaces_agrees_with_q2():
    """A quadratic displacement field lies in both the serendipity and the Q2
    spaces: on a flat mesh (where both geometry maps are the same affine map)
    the 20-node centre stresses equal the Q2 ones of oracle.fem."""
    lam = block(3, 2, [(2, 0.5, 0, 30.0), (1, 0.05, 1, 0.0)], sx=[0.0, 0.8, 1.5, 2.4], sy=[0.0, 1.1, 2.0])
    m = serendipity.Mesh20(lam)
    rng = np.random.default_rng(9)
    A = rng.standard_normal((3, 3)) * 1e-3
    B = rng.standard_normal((3, 3)) * 1e-4

    def field(X):
        return X @ A.T + (X[:, [0]] * X[:, [1]]) @ B[:, :1].T + (X[:, [2]] ** 2) @ B[:, 1:2].T

    s20, t20 = serendipity.stress_slr20(m, field(m.X).ravel())
    q2 = fem.Mesh(lam)
    s2, t2 = fem.stress_slr(q2, field(q2.X).ravel())
    assert np.abs(s20 - s2).max() <= 1e-11 * np.abs(s2).max()
    assert np.abs(t20 - t2).max() <= 1e-11 * np.abs(t2).max()

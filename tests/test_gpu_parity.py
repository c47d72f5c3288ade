"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Tolerances (FP64 everywhere unless stated):
  * K u, loads, stresses: pure FP64 arithmetic in a different order, 1e-12
    relative (a few hundred roundings per entry);
  * local Dirichlet solves: both sides are direct solves of the same SPD
    matrices; the difference is bounded by cond(A_j) * eps, cond(A_j) about
    1e6-1e8 for these laminates, so 1e-8 relative;
  * GenEO eigenvalues: the GPU subspace iteration stops when the Ritz values
    change by less than 1e-10 relative between iterations, 1e-7 relative;
  * u against the oracle's direct solve: 1e-8 relative (the required bar);
  * iteration counts: within 15% of the oracle's PCG.
"""
import numpy as np
import pytest

from oracle import fem, geneo
from paper_1707_04228_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def lib_mod(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    return lib


def small_flat():
    lam = inputs.flat_plate_c0()
    lam.sv = np.linspace(0.0, 20.0, 6)       # ragged: 5 elements over 2 subdomains
    lam.lv = np.array([0.0, 3.0, 8.0, 20.0])
    lam.layer_nel = [1, 1, 1, 1, 1, 1, 1]
    lam.dir_dof, lam.dir_val = inputs.clamp_face(lam, inputs.FACE_SM)
    lam.theta = inputs.gaussian_theta(lam, 8.0, 4.0)
    lam.px, lam.py, lam.pz, lam.nev = 2, 2, 1, 8
    return lam


def small_curved():
    lam = inputs.corner_mini(n_arc=5, n_limb=1, n_width=3, nel_layer=1, angles=(0, 45, 90), nsub=(3, 1, 1), nev=8,
                             limb_L=3.0, width=3.0)
    return lam


@pytest.fixture(scope="module", params=["flat", "curved"])
def case(request, lib_mod):
    lam = small_flat() if request.param == "flat" else small_curved()
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    s = lib_mod.Solver.from_laminate(lam)
    return lam, mesh, sysm, s


def test_ku_matches_assembled_oracle(case):
    lam, mesh, sysm, s = case
    x = inputs.random_vector(mesh.n_dof, 11)
    y = s.apply_K(x)
    assert rel(y, sysm.K @ x) <= 1e-12


def test_ku_device_pointers(case):
    import torch
    lam, mesh, sysm, s = case
    x = torch.from_numpy(inputs.random_vector(mesh.n_dof, 12)).cuda()
    y = torch.empty_like(x)
    s.apply_K(x, out=y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), sysm.K @ x.cpu().numpy()) <= 1e-12


def test_traction_loads(case):
    lam, mesh, sysm, s = case
    f = s.rhs()
    if lam.traction:
        assert rel(f, sysm.f) <= 1e-13
    else:
        assert np.abs(f).max() == 0.0


def test_stress_recovery(case):
    lam, mesh, sysm, s = case
    u = inputs.random_vector(mesh.n_dof, 13) * 1e-3
    s33, t13, peak = s.stress(u)
    r33, r13 = fem.stress_slr(mesh, u)
    assert rel(s33, r33) <= 1e-11 and rel(t13, r13) <= 1e-11
    assert abs(peak - r33[mesh.is_resin].max()) <= 1e-11 * np.abs(r33).max()


def test_one_level_schwarz_matches_oracle(lib_mod):
    lam = small_flat()
    sysm = fem.System(fem.Mesh(lam))
    dec = geneo.Decomposition(sysm, lam.px, lam.py, lam.pz, 1)
    P1 = geneo.GenEO(dec, 0, coarse=False)
    s = lib_mod.Solver.from_laminate(lam, nev=0)
    r = inputs.random_vector(sysm.mesh.n_dof, 14)
    r[sysm.is_dir] = 0.0
    z = s.apply_prec(r)
    zr = P1.apply(r[sysm.free])
    assert rel(z[sysm.free], zr) <= 1e-8
    assert np.abs(z[sysm.is_dir]).max() == 0.0


def test_geneo_eigenvalues_and_two_level_prec(lib_mod):
    lam = small_flat()
    sysm = fem.System(fem.Mesh(lam))
    dec = geneo.Decomposition(sysm, lam.px, lam.py, lam.pz, 1)
    P = geneo.GenEO(dec, lam.nev, eig_method="dense")
    s = lib_mod.Solver.from_laminate(lam)
    ev = s.geneo_eigenvalues().reshape(len(dec.subs), lam.nev)
    ref = np.array(P.eigvals)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(ev - ref) <= 1e-7 * scale)
    # the coarse space spans the same subspaces, so the two-level operators agree
    r = inputs.random_vector(sysm.mesh.n_dof, 15)
    r[sysm.is_dir] = 0.0
    assert rel(s.apply_prec(r)[sysm.free], P.apply(r[sysm.free])) <= 1e-6


@pytest.mark.parametrize("which", ["flat", "curved"])
def test_full_solve_matches_direct_oracle(lib_mod, which):
    lam = small_flat() if which == "flat" else small_curved()
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    u_ref = sysm.direct()
    _, it_ref, _, _, _ = geneo.solve(lam, system=sysm)
    s = lib_mod.Solver.from_laminate(lam)
    u, info = s.solve()
    assert info["status"] == 0
    assert rel(u, u_ref) <= 1e-8
    assert info["rel_resid"] <= lam.tol
    assert abs(info["iters"] - it_ref) <= max(2, 0.15 * it_ref)
    s33, _, peak = s.stress(u)
    r33, _ = fem.stress_slr(mesh, u_ref)
    assert abs(peak - r33[mesh.is_resin].max()) <= 1e-6 * np.abs(r33).max()


def test_flat_plate_c0_full(lib_mod):
    """8x8x14 [0/90]s plate, 2x2x2 subdomains, 8 eigenvectors, PCG to 1e-10."""
    lam = inputs.flat_plate_c0()
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    u_ref = sysm.direct()
    s = lib_mod.Solver.from_laminate(lam)
    u, info = s.solve()
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    assert rel(u, u_ref) <= 1e-8
    s33, _, peak = s.stress(u)
    r33, _ = fem.stress_slr(mesh, u_ref)
    assert abs(peak - r33[mesh.is_resin].max()) <= 1e-6 * np.abs(r33).max()


def test_mixed_precision_solve(lib_mod):
    lam = small_flat()
    sysm = fem.System(fem.Mesh(lam))
    u_ref = sysm.direct()
    s = lib_mod.Solver.from_laminate(lam, precision=lib_mod.GL_PREC_MIXED, tol=1e-10)
    u, info = s.solve()
    assert info["status"] == 0
    assert info["rel_resid_true"] <= 1e-8
    assert rel(u, u_ref) <= 1e-6


def test_error_paths(lib_mod):
    lam = small_flat()
    s = lib_mod.Solver.from_laminate(lam, max_iter=2)
    u, info = s.solve(check=False)
    assert info["status"] == -5 and info["iters"] == 2
    f = s.rhs()
    f[10] = np.nan
    with pytest.raises(lib_mod.GLError) as e:
        s.solve(f)
    assert e.value.code == -6
    with pytest.raises(lib_mod.GLError):
        lib_mod.Solver.from_laminate(lam, overlap=0)


def test_single_subdomain_is_a_direct_solve(lib_mod):
    lam = small_flat()
    s = lib_mod.Solver.from_laminate(lam, px=1, py=1, pz=1, nev=0)
    u, info = s.solve()
    assert info["iters"] <= 2
    u_ref = fem.System(fem.Mesh(lam)).direct()
    assert rel(u, u_ref) <= 1e-9


def test_failure_index_matches_oracle(lib_mod):
    """Eq. eq-Camanho on the resin interfaces of a loaded curved corner."""
    lam = small_curved()
    mesh = fem.Mesh(lam)
    u = fem.System(mesh).direct()
    s = lib_mod.Solver.from_laminate(lam)
    F, peak, e = s.failure_index(u)
    ref = fem.failure_index(mesh, u)
    assert rel(F, ref) <= 1e-11
    assert np.all(F[~mesh.is_resin] == 0.0)
    assert abs(peak - ref.max()) <= 1e-11 * ref.max() + 2e-5 * ref.max()
    assert F[e] == peak and mesh.is_resin[e]


def test_coincident_subdomains_drop_coarse_columns(lib_mod):
    """Two elements across the width split in two with overlap 1: each pair of
    subdomains coincides and their GenEO vectors span the same space (up to the
    eigensolver's convergence), so K_0 is singular.  The dependent columns are
    dropped (at most the 2 x 6 of the oracle, which finds the exact duplicates)
    and the solve still reaches the direct solution."""
    lam = inputs.corner_mini(n_arc=4, n_limb=1, n_width=2, nel_layer=1, angles=(0, 90), nsub=(2, 2, 1), nev=6,
                             limb_L=2.0, width=2.0)
    mesh = fem.Mesh(lam)
    u_ref = fem.System(mesh).direct()
    s = lib_mod.Solver.from_laminate(lam, px=2, py=2, pz=1, nev=6, tol=1e-12)
    u, info = s.solve()
    assert info["status"] == 0
    assert 0 < info["n_coarse_dropped"] <= 12
    assert rel(u, u_ref) <= 1e-8


def wrinkled_corner():
    """Mini curved corner carrying the paper's sech^2 geometric wrinkle (Section 3,
    Eq. eq-f) instead of a misalignment field: nodes moved through the thickness,
    fibre angles following the deformed plies."""
    lam = inputs.corner_mini(n_arc=6, n_limb=1, n_width=4, nel_layer=2, angles=(0, 90), nsub=(3, 2, 1), nev=8,
                             limb_L=2.0, width=4.0)
    lam.node_dr, lam.theta = inputs.sech2_wrinkle(lam, 0.05)
    return lam


def test_wrinkled_corner_matches_oracle(lib_mod):
    lam = wrinkled_corner()
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    s = lib_mod.Solver.from_laminate(lam)
    x = inputs.random_vector(mesh.n_dof, 17)
    assert rel(s.apply_K(x), sysm.K @ x) <= 1e-12
    u_ref = sysm.direct()
    u, info = s.solve()
    assert info["status"] == 0 and rel(u, u_ref) <= 1e-8
    _, _, peak = s.stress(u)
    r33, _ = fem.stress_slr(mesh, u_ref)
    assert abs(peak - r33[mesh.is_resin].max()) <= 1e-6 * np.abs(r33).max()


def test_folding_wrinkle_is_rejected(lib_mod):
    lam = wrinkled_corner()
    lam.node_dr, lam.theta = inputs.sech2_wrinkle(lam, 2.0)     # larger than the thickness allows
    with pytest.raises(lib_mod.GLError) as e:
        lib_mod.Solver.from_laminate(lam)
    assert e.value.code == -1


def edge_resin_corner():
    """Mini curved corner whose outermost element columns across the width are
    resin in every layer (per-element materials, as the paper's edge strips)."""
    lam = inputs.corner_mini(n_arc=6, n_limb=1, n_width=5, nel_layer=1, angles=(0, 45, 90), nsub=(3, 1, 1), nev=8,
                             limb_L=2.0, width=5.0)
    em = np.broadcast_to(np.asarray(lam.layer_mat)[lam.elem_layer()][:, None, None], (lam.nz, lam.ny, lam.nx)).copy()
    em[:, 0, :] = 1
    em[:, -1, :] = 1
    lam.elem_mat = em
    return lam


def test_edge_resin_corner_matches_oracle(lib_mod):
    import torch
    from oracle import adjoint
    from paper_1707_04228_gb300.autograd import pnorm, stress_of_theta
    lam = edge_resin_corner()
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    assert mesh.is_resin.reshape(lam.nz, lam.ny, lam.nx)[:, 0, :].all()
    s = lib_mod.Solver.from_laminate(lam, tol=1e-12)
    x = inputs.random_vector(mesh.n_dof, 19)
    assert rel(s.apply_K(x), sysm.K @ x) <= 1e-12
    u_ref = sysm.direct()
    u, info = s.solve()
    assert info["status"] == 0 and rel(u, u_ref) <= 1e-8
    _, _, peak = s.stress(u)
    r33, _ = fem.stress_slr(mesh, u_ref)
    assert abs(peak - r33[mesh.is_resin].max()) <= 1e-6 * np.abs(r33).max()
    # the adjoint contraction reads the same per-element materials
    mask = inputs.arc_resin_mask(lam) & mesh.is_resin
    theta = torch.tensor(mesh.theta, dtype=torch.float64, device="cuda", requires_grad=True)
    J = pnorm(stress_of_theta(theta, s), torch.tensor(mask, device="cuda"), 8)
    J.backward()
    J_ref, g_ref, _ = adjoint.gradient(sysm, mask, 8)
    assert abs(J.item() - J_ref) <= 1e-9 * J_ref
    assert np.abs(theta.grad.cpu().numpy() - g_ref).max() <= 1e-6 * np.abs(g_ref).max()

"""Periodic width conditions (Section 3, the 39-ply study) on the GPU against
the oracle's direct solve with the last width plane identified with the
first (fem.periodic_width_direct, pinned against the generalised
plane-strain field of a stretched strip in test_oracle_pins.py).

The library keeps the full node grid: the last plane's entries are not
unknowns (ignored on input, returned equal to the first plane's by the
solve, zero in K u).  Every subdomain spans the width (py = 1), the first
width plane being the root separator of its dissection.

Tolerances as in test_gpu_parity.py: K u 1e-12; u against the direct solve
1e-8 (PCG to 1e-10); centre stresses of the solution 1e-7.
"""
import numpy as np
import pytest

from oracle import fem
from paper_1707_04228_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def lib_mod(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    return lib


def flat():
    lam = inputs.flat_plate_c0()
    lam.sv = np.linspace(0.0, 20.0, 7)
    lam.lv = np.array([0.0, 4.0, 9.0, 14.0, 20.0])
    lam.layer_nel = [1] * 7
    lam.dir_dof, lam.dir_val = inputs.clamp_face(lam, inputs.FACE_SM)
    lam.theta = inputs.gaussian_theta(lam, 8.0, 4.0)
    lam.px, lam.py, lam.pz, lam.nev = 3, 1, 1, 8
    lam.periodic_width = 1
    return lam


def curved():
    lam = inputs.corner_mini(n_arc=5, n_limb=1, n_width=3, nel_layer=1, angles=(0, 45, 90), nsub=(3, 1, 1), nev=8,
                             limb_L=3.0, width=3.0)
    lam.periodic_width = 1
    return lam


def slave_mask(mesh):
    iy = (np.arange(mesh.n_nodes) // mesh.NX) % mesh.NY
    return np.repeat(iy == mesh.NY - 1, 3)


def partner(mesh):
    node = np.arange(mesh.n_nodes)
    iy = (node // mesh.NX) % mesh.NY
    rep = np.where(iy == mesh.NY - 1, node - (mesh.NY - 1) * mesh.NX, node)
    return (3 * rep[:, None] + np.arange(3)[None, :]).ravel()


@pytest.fixture(scope="module", params=["flat", "curved"])
def case(request, lib_mod):
    lam = flat() if request.param == "flat" else curved()
    mesh = fem.Mesh(lam)
    K = fem.assemble_K(mesh)
    s = lib_mod.Solver.from_laminate(lam)
    return lam, mesh, K, s


def test_ku_is_the_identified_operator(case):
    """K_p = A^T K A: x taken equal on both planes, K x folded onto the first plane."""
    lam, mesh, K, s = case
    sl, rep = slave_mask(mesh), partner(mesh)
    x = inputs.random_vector(mesh.n_dof, 71)
    xin = x.copy()
    xin[sl] = inputs.random_vector(int(sl.sum()), 72)   # ignored by the library
    y = s.apply_K(xin)
    xp = x[rep]                                         # the periodic field
    yr = K @ xp
    yref = np.zeros_like(yr)
    np.add.at(yref, rep, yr)                            # A^T (K A x)
    assert rel(y, yref) <= 1e-12
    assert np.abs(y[sl]).max() == 0.0


def test_solve_matches_the_periodic_direct_solve(case):
    lam, mesh, K, s = case
    u_ref = fem.periodic_width_direct(mesh, lam.dir_dof, lam.dir_val, K=K)
    u, info = s.solve()
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    assert rel(u, u_ref) <= 1e-8
    sl, rep = slave_mask(mesh), partner(mesh)
    assert np.array_equal(u[sl], u[rep][sl])             # the last plane returned equal to the first
    s33, t13, _ = s.stress(u)
    r33, r13 = fem.stress_slr(mesh, u_ref)
    assert rel(s33, r33) <= 1e-7 and rel(t13, r13) <= 1e-7


def test_periodic_width_needs_one_subdomain_across(lib_mod):
    with pytest.raises(lib_mod.GLError) as e:
        lib_mod.Solver.from_laminate(flat(), py=2)
    assert e.value.code == -1
    lam = flat()
    lam.element = 1
    with pytest.raises(lib_mod.GLError) as e:
        lib_mod.Solver.from_laminate(lam)
    assert e.value.code == -1

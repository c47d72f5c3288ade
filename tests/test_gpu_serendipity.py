"""The 20-node serendipity element on the GPU against the oracle's serendipity
element (oracle/serendipity.py, assembled independently from its own shape
functions and numbering).

The library keeps the Q2 node grid for the serendipity mesh: its unknowns are
the grid nodes with at most one odd index, and the face- and body-centre
entries of its vectors are not unknowns (ignored on input, returned as the
serendipity field's values by the solve, zero in K u and the loads).  The
parity cases put random values there on input to check that they are ignored.

Tolerances as for Q2 (test_gpu_parity.py): K u, loads 1e-12 / 1e-13 relative;
centre stresses 1e-11; the solution of the plate against the oracle's direct
solve 1e-8 (PCG to 1e-10).
"""
import numpy as np
import pytest

from oracle import serendipity
from paper_1707_04228_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def lib_mod(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    return lib


def plate_c0():
    """The 8x8x14 [0/90]s plate in serendipity elements: 13,527 DOF."""
    lam = inputs.flat_plate_c0()
    lam.element = 1
    return lam


def curved():
    lam = inputs.corner_mini(n_arc=5, n_limb=1, n_width=3, nel_layer=1, angles=(0, 45, 90), nsub=(3, 1, 1), nev=8,
                             limb_L=3.0, width=3.0)
    lam.element = 1
    return lam


def embed(m20, v20, junk_seed):
    """A Q2-grid vector with v20 on the serendipity nodes and random values elsewhere."""
    out = inputs.random_vector(3 * m20.q2.n_nodes, junk_seed)
    d = (3 * m20.q2_of[:, None] + np.arange(3)[None, :]).ravel()
    out[d] = v20
    return out, d


@pytest.fixture(scope="module", params=["flat", "curved"])
def case(request, lib_mod):
    lam = plate_c0() if request.param == "flat" else curved()
    m20 = serendipity.Mesh20(lam)
    K20 = m20.assemble_K()
    s = lib_mod.Solver.from_laminate(lam)
    return lam, m20, K20, s


def test_ku_matches_the_oracle_serendipity_assembly(case):
    lam, m20, K20, s = case
    x20 = inputs.random_vector(m20.n_dof, 61)
    x, d = embed(m20, x20, 62)
    y = s.apply_K(x)
    assert rel(y[d], K20 @ x20) <= 1e-12
    slave = np.ones(y.size, bool)
    slave[d] = False
    assert np.abs(y[slave]).max() == 0.0


def test_loads_and_centre_stresses(case):
    lam, m20, K20, s = case
    _, d = embed(m20, np.zeros(m20.n_dof), 63)
    f = s.rhs()
    f_ref = sum((serendipity.traction_load20(m20, face, t) for face, t in lam.traction), np.zeros(m20.n_dof))
    if lam.traction:
        assert rel(f[d], f_ref) <= 1e-13
    u20 = inputs.random_vector(m20.n_dof, 64) * 1e-3
    u, _ = embed(m20, u20, 65)
    s33, t13, _ = s.stress(u)
    r33, r13 = serendipity.stress_slr20(m20, u20)
    assert rel(s33, r33) <= 1e-11 and rel(t13, r13) <= 1e-11


def test_plate_solve_matches_the_oracle_direct_solve(lib_mod):
    lam = plate_c0()
    m20 = serendipity.Mesh20(lam)
    K20 = m20.assemble_K()
    f20 = sum((serendipity.traction_load20(m20, face, t) for face, t in lam.traction), np.zeros(m20.n_dof))
    # the clamp in serendipity numbering: its DOFs on serendipity nodes
    node20 = m20.of_q2[np.asarray(lam.dir_dof) // 3]
    keep = node20 >= 0
    dir20 = 3 * node20[keep] + np.asarray(lam.dir_dof)[keep] % 3
    u_ref = serendipity.solve_dirichlet(m20, K20, f20, dir20, np.asarray(lam.dir_val)[keep])
    s = lib_mod.Solver.from_laminate(lam)
    u, info = s.solve()
    _, d = embed(m20, np.zeros(m20.n_dof), 66)
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    assert info["n_free"] == m20.n_dof - dir20.size
    assert rel(u[d], u_ref) <= 1e-8
    # the face- and body-centre entries carry the serendipity field: its stresses from the returned vector
    s33, _, _ = s.stress(u)
    r33, _ = serendipity.stress_slr20(m20, u_ref)
    assert rel(s33, r33) <= 1e-7


def test_batch_rejects_the_serendipity_element(lib_mod):
    with pytest.raises(lib_mod.GLError) as e:
        lib_mod.Batch([plate_c0()])
    assert e.value.code == -1

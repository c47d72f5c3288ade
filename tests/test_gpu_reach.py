"""GPU parity on a laminate that takes the code paths of the full-size runs.

The parity cases of test_gpu_parity.py are small enough that every level of
their dissection trees has fewer fronts than the launch threshold at which the
local sweeps switch from 512- to 256-thread blocks (1,216 fronts), their local
factors fit one workspace group, and the GenEO eigensolver treats all
subdomains in one group.  The full-size corner takes the other branches.  This
curved corner (32 x 8 x 7 Q2 elements, [0/90]s with resin interfaces, 49,725
DOF) is split into 32 x 8 in-plane subdomains, so that one level of its
dissection trees holds 1,260 fronts, more than the threshold (the other
levels stay below it: both launch shapes run), and the workspace budgets of
gl_opts force one subdomain per factorisation group and per eigensolver
group.

Tolerances as in test_gpu_parity.py: u against the oracle's direct solve to
1e-8 (FP64, PCG to 1e-10) and 1e-6 (mixed, true residual 1e-8); the residual
of the GPU solution measured with the oracle's own assembled K; the one-level
Schwarz operator against the oracle's (both direct local solves) to 1e-8.
"""
import numpy as np
import pytest

from oracle import fem, geneo
from paper_1707_04228_gb300 import inputs

pytestmark = pytest.mark.gpu

WIDE_SWEEP_BELOW = 1216     # fronts per level under which the sweeps use 512-thread blocks


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def reach_corner():
    return inputs.curved_corner(n_arc=24, n_limb=4, n_width=8, nel_layer=1, angles=(0, 90), nsub=(32, 8, 1),
                                nev=10, name="curved_corner_reach_32x8x7")


@pytest.fixture(scope="module")
def lib_mod(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    return lib


@pytest.fixture(scope="module")
def oracle_case():
    lam = reach_corner()
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    return lam, mesh, sysm, sysm.direct()


def oracle_residual(sysm, u):
    """||f - K u|| / ||f|| on the free DOFs with the oracle's assembled K."""
    return np.linalg.norm(sysm.ff - sysm.Kff @ u[sysm.free]) / np.linalg.norm(sysm.ff)


@pytest.fixture(scope="module")
def fp64_run(lib_mod, oracle_case):
    lam = oracle_case[0]
    s = lib_mod.Solver.from_laminate(lam)
    u, info = s.solve()
    return s, u, info


def test_fp64_solve_takes_the_full_size_sweep_branch(fp64_run, oracle_case):
    lam, mesh, sysm, u_ref = oracle_case
    s, u, info = fp64_run
    prof = s.profile_read()
    assert prof["max_level_fronts"] >= WIDE_SWEEP_BELOW
    assert prof["factor_groups"] == 1 and prof["eig_groups"] == 1
    assert info["status"] == 0 and info["rel_resid"] <= 1e-10
    assert oracle_residual(sysm, u) <= 1e-9
    assert rel(u, u_ref) <= 1e-8
    _, _, peak = s.stress(u)
    r33, _ = fem.stress_slr(mesh, u_ref)
    assert abs(peak - r33[mesh.is_resin].max()) <= 1e-6 * np.abs(r33).max()


def test_one_subdomain_per_group(lib_mod, oracle_case, fp64_run):
    """Budgets of one byte: every subdomain is its own factorisation group and
    its own eigensolver group.  The factors are the same, the coarse space the
    same within the eigensolver's convergence, so the solution still matches."""
    lam, mesh, sysm, u_ref = oracle_case
    s = lib_mod.Solver.from_laminate(lam, factor_ws_bytes=1.0, eig_group_bytes=1.0)
    prof = s.profile_read()
    assert prof["factor_groups"] == prof["n_sub"] == 256
    assert prof["eig_groups"] == 256
    u, info = s.solve()
    assert info["status"] == 0
    assert rel(u, u_ref) <= 1e-8
    assert oracle_residual(sysm, u) <= 1e-9
    it0 = fp64_run[2]["iters"]
    assert abs(info["iters"] - it0) <= max(2, 0.15 * it0)


def test_one_level_schwarz_at_reach(lib_mod, oracle_case):
    lam, mesh, sysm, _ = oracle_case
    dec = geneo.Decomposition(sysm, lam.px, lam.py, lam.pz, 1)
    P1 = geneo.GenEO(dec, 0, coarse=False)
    s = lib_mod.Solver.from_laminate(lam, nev=0, factor_ws_bytes=2e6)
    assert s.profile_read()["factor_groups"] > 1
    r = inputs.random_vector(mesh.n_dof, 41)
    r[sysm.is_dir] = 0.0
    z = s.apply_prec(r)
    assert rel(z[sysm.free], P1.apply(r[sysm.free])) <= 1e-8


def test_mixed_precision_at_reach(lib_mod, oracle_case):
    lam, mesh, sysm, u_ref = oracle_case
    s = lib_mod.Solver.from_laminate(lam, precision=lib_mod.GL_PREC_MIXED, tol=1e-8)
    assert s.profile_read()["max_level_fronts"] >= WIDE_SWEEP_BELOW
    u, info = s.solve()
    assert info["status"] == 0
    assert info["rel_resid_true"] <= 1e-8
    assert oracle_residual(sysm, u) <= 1.05e-8
    assert rel(u, u_ref) <= 1e-6

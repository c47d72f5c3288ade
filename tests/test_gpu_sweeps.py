"""GPU parity of the local triangular solves in their launch forms.

The sweeps with the local factors treat each front's panel as a triangle (its
pivot rows, in partitioned-inverse form) over a rectangle (its structure
rows): the backward sweep forms the rectangle's transposed product for all
pivot columns at once, then the triangle block by block, a short last block
read 16, 8 or 4 columns wide.  With gl_opts.sweep_overlap the two halves of
the subdomains sweep on their own streams.  The ragged corner below has
fronts of many sizes, short last blocks of every width and fronts with fewer
32-column blocks than warps (several warps per block of the rectangle).

Tolerances: the one-level Schwarz operator (direct local solves) against the
oracle's to 1e-8, as in test_gpu_parity.py; the GenEO eigenvalues, whose
eigensolver sweeps four right-hand sides at once, against the oracle's dense
LAPACK to 1e-7; u against the oracle's direct solve to 1e-8; the overlapped
sweeps against the sequential ones to 1e-13 (the same products; only the
forward sweep's atomic additions into rows shared by sibling fronts may land
in another order).
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


def ragged_corner():
    # 3 x 2 in-plane subdomains of unequal size, plies and resin: fronts of
    # many sizes, none a multiple of 32 rows in general
    return inputs.corner_mini(n_arc=7, n_limb=1, n_width=3, nel_layer=1, angles=(0, 45, 90), nsub=(3, 2, 1),
                              nev=8, limb_L=3.0, width=3.0)


@pytest.fixture(scope="module")
def oracle_case():
    lam = ragged_corner()
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    return lam, mesh, sysm


def test_one_level_schwarz(lib_mod, oracle_case):
    lam, mesh, sysm = oracle_case
    dec = geneo.Decomposition(sysm, lam.px, lam.py, lam.pz, 1)
    P1 = geneo.GenEO(dec, 0, coarse=False)
    r = inputs.random_vector(mesh.n_dof, 57)
    r[sysm.is_dir] = 0.0
    s = lib_mod.Solver.from_laminate(lam, nev=0)
    assert rel(s.apply_prec(r)[sysm.free], P1.apply(r[sysm.free])) <= 1e-8


def test_eigenvalues_and_solve(lib_mod, oracle_case):
    lam, mesh, sysm = oracle_case
    dec = geneo.Decomposition(sysm, lam.px, lam.py, lam.pz, 1)
    P = geneo.GenEO(dec, lam.nev, eig_method="dense")
    s = lib_mod.Solver.from_laminate(lam)
    ev = s.geneo_eigenvalues().reshape(len(dec.subs), lam.nev)
    ref = np.array(P.eigvals)
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(ev - ref) <= 1e-7 * scale)
    u, info = s.solve()
    assert info["status"] == 0
    assert rel(u, sysm.direct()) <= 1e-8


def test_overlapped_halves(lib_mod, oracle_case):
    """gl_opts.sweep_overlap: the two halves of the subdomains sweep on their
    own streams (top levels at high priority)."""
    lam, mesh, sysm = oracle_case
    r = inputs.random_vector(mesh.n_dof, 59)
    r[sysm.is_dir] = 0.0
    zs = {}
    for ov in (-1, 2, 40):
        s = lib_mod.Solver.from_laminate(lam, sweep_overlap=ov)
        zs[ov] = s.apply_prec(r)
    assert rel(zs[2], zs[-1]) <= 1e-13
    assert rel(zs[40], zs[-1]) <= 1e-13     # every level counted as top: one stream per half
    u, info = s.solve()
    assert info["status"] == 0
    assert rel(u, sysm.direct()) <= 1e-8


def test_level_profile(lib_mod, oracle_case):
    """gl_profile_levels: per-level sizes add up to the plan's totals, and the
    timed sweeps cover every level that has fronts; with phase timing only
    (gl_profile 1) no level is timed."""
    lam, mesh, sysm = oracle_case
    s = lib_mod.Solver.from_laminate(lam)
    s.profile(2)
    s.solve()
    prof = s.profile_read()
    lv = s.profile_levels()
    s.profile(False)
    assert lv["calls"] >= 1
    assert lv["nonzeros"].sum() == prof["factor_nonzeros"]
    assert np.all(lv["padded"] >= lv["nonzeros"])
    has = lv["fronts"] > 0
    assert np.all(lv["fwd_ms"][has] > 0) and np.all(lv["bwd_ms"][has] > 0)
    assert np.all(lv["max_front"][has] > 0)
    s.profile(1)
    s.solve()
    assert s.profile_levels()["calls"] == 0
    assert s.profile_read()["n_local"] >= 1
    s.profile(False)

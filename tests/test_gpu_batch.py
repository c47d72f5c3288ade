"""Batched solve of several laminates of different sizes and stacks in one
engine (one launch per phase, graph-replayed iterations) against the same
laminates solved one by one and against the oracle's direct solves.

Tolerances: u against the direct solve 1e-8 relative (the bar for FP64);
iteration counts equal to the single-laminate solves with the same
decomposition up to one iteration (atomics change rounding order only).
"""
import numpy as np
import pytest

from oracle import fem
from paper_1707_04228_gb300 import inputs

pytestmark = pytest.mark.gpu


def laminates():
    rng = np.random.default_rng(4228)
    out = [inputs.flat_random(rng, n, P, amp, nsub=(2, 2, 1), nev=6, name=f"p{i}")
           for i, (n, P, amp) in enumerate([(4, 3, 5.0), (6, 4, 0.0), (5, 2, 11.0)])]
    out.append(inputs.corner_mini(n_arc=4, n_limb=1, n_width=2, nel_layer=1, angles=(0, 90), nsub=(2, 2, 1), nev=6,
                                  limb_L=2.0, width=2.0))
    return out


def test_batch_matches_single_and_oracle(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    lams = laminates()
    b = lib.Batch(lams)
    b.setup(px=2, py=2, nev=6, tol=1e-10)
    us, infos = b.solve()
    assert (b.grid() == 2).all()
    for lam, u, info in zip(lams, us, infos):
        assert info["status"] == 0 and info["rel_resid"] <= 1e-10
        ref = fem.System(fem.Mesh(lam)).direct()
        assert np.linalg.norm(u - ref) <= 1e-8 * np.linalg.norm(ref)
        single = lib.Solver.from_laminate(lam, px=2, py=2, pz=1, nev=6)
        _, si = single.solve()
        assert abs(si["iters"] - info["iters"]) <= 1
    # a second solve replays the captured graph and gives the same answer
    us2, infos2 = b.solve()
    for u, u2 in zip(us, us2):
        assert np.linalg.norm(u - u2) <= 1e-12 * np.linalg.norm(u)
    b.close()


def test_batch_autotuned_mixed(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    lams = inputs.batch_plates(count=3, dof_lo=20_000, dof_hi=60_000, seed=7)
    b = lib.Batch(lams)
    b.setup(px=0, py=0, nev=6, tol=1e-8, precision=lib.GL_PREC_MIXED)
    g = b.grid()
    assert all(8 <= px * py <= 64 for px, py in g)
    us, infos = b.solve()
    for lam, u, info in zip(lams, us, infos):
        assert info["status"] == 0 and info["rel_resid_true"] <= 1e-7
        ref = fem.System(fem.Mesh(lam)).direct()
        assert np.linalg.norm(u - ref) <= 1e-5 * np.linalg.norm(ref)
    b.close()

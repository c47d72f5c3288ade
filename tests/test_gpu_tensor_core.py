"""FP32 local factors with the trailing updates on the tensor cores.

In the mixed-precision form the local factorisation is FP32; its rank-128
trailing updates run on tcgen05 with TF32 operands split into hi + lo parts
(FP32-level products, FP32 accumulation).  With one subdomain and no coarse
space the preconditioner is the direct solve of the whole K_ff, so its
residual measured with the oracle's assembled K_ff shows the factor's
accuracy independently of the CUDA path.  An FP32 factor of these laminates
(0.02 mm resin layers, strongly anisotropic plies) leaves a relative residual
of order eps_32 x cond, about 1e-2, where the FP64 factor leaves 1e-10: the
bar is therefore the FP32 factor with the rank-32 updates on the FP32 CUDA
cores.  The split keeps about 22 of FP32's 24 significant bits per product,
so the tensor-core factor must be within a factor 4 of it -- and far from the
garbage a wrong operand layout would give.  The two FP32 factors
round differently, so they are compared by residual, not element by element.
"""
import numpy as np
import pytest

from oracle import fem
from paper_1707_04228_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_mod(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    return lib


def residual(sysm, z, r):
    return np.linalg.norm(sysm.Kff @ z[sysm.free] - r[sysm.free]) / np.linalg.norm(r[sysm.free])


@pytest.mark.parametrize("case", ["flat_c0", "curved"])
def test_fp32_direct_solve_residual_with_tensor_core_updates(lib_mod, case):
    if case == "flat_c0":
        lam = inputs.flat_plate_c0()          # fronts of up to ~900 rows: several 128-column panels
    else:
        lam = inputs.corner_mini(n_arc=6, n_limb=1, n_width=4, nel_layer=2, angles=(0, 45, -45, 90), nsub=(1, 1, 1))
    mesh = fem.Mesh(lam)
    sysm = fem.System(mesh)
    r = inputs.random_vector(mesh.n_dof, 51)
    r[sysm.is_dir] = 0.0
    res = {}
    for key, kw in (("fp64", dict(precision=lib_mod.GL_PREC_FP64)),
                    ("tc", dict(precision=lib_mod.GL_PREC_MIXED, fp32_update=0)),
                    ("cuda_core", dict(precision=lib_mod.GL_PREC_MIXED, fp32_update=1))):
        s = lib_mod.Solver.from_laminate(lam, px=1, py=1, pz=1, nev=0, **kw)
        z = s.apply_prec(r)
        assert np.all(np.isfinite(z)) and np.abs(z[sysm.is_dir]).max() == 0.0
        res[key] = residual(sysm, z, r)
        s.close()
    print(case, res)
    assert res["fp64"] <= 1e-9
    assert res["cuda_core"] <= 0.1
    assert res["tc"] <= 4.0 * res["cuda_core"]


def test_mixed_solve_with_cuda_core_updates_matches(lib_mod):
    """The full mixed-precision solve reaches the same answer with either update."""
    lam = inputs.flat_plate_c0()
    lam.px, lam.py, lam.pz = 2, 2, 1
    sysm = fem.System(fem.Mesh(lam))
    u_ref = sysm.direct()
    its = {}
    for upd in (0, 1):
        s = lib_mod.Solver.from_laminate(lam, precision=lib_mod.GL_PREC_MIXED, tol=1e-8, fp32_update=upd)
        u, info = s.solve()
        assert info["status"] == 0 and info["rel_resid_true"] <= 1e-8
        assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) <= 1e-6
        its[upd] = info["iters"]
        s.close()
    assert abs(its[0] - its[1]) <= 2

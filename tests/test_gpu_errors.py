"""Error paths of the C ABI that need the GPU, raised from the host side.

* GL_ERR_NOT_SPD: an orthotropic material with positive moduli but Poisson
  ratios that make its compliance indefinite (1 - 2 nu^2 ... < 0) passes the
  material checks; the local factorisation meets a non-positive pivot and
  gl_setup reports it.  The kernels substitute a unit pivot and raise a flag,
  so nothing faults.
* GL_ERR_OOM: device memory is taken by the test before gl_setup, leaving
  16 MB, less than the local factors need; the allocation failure comes back
  as GL_ERR_OOM, and once the memory is returned the same device serves a
  normal setup.
"""
import numpy as np
import pytest

from paper_1707_04228_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib_mod(gl_lib, cuda_ok):
    from paper_1707_04228_gb300 import lib
    return lib


def plate():
    lam = inputs.flat_plate_c0()
    lam.px, lam.py, lam.pz = 2, 2, 1
    return lam


def test_indefinite_material_reports_not_spd(lib_mod):
    lam = plate()
    bad = dict(inputs.PLY_T1)
    bad.update(E1=10000.0, E2=10000.0, E3=10000.0, nu12=0.9, nu13=0.9, nu23=0.9)
    S = np.zeros((3, 3))
    S[np.diag_indices(3)] = 1.0 / 10000.0
    S[0, 1] = S[1, 0] = S[0, 2] = S[2, 0] = S[1, 2] = S[2, 1] = -0.9 / 10000.0
    assert np.linalg.eigvalsh(S).min() < 0.0          # the normal-stress compliance is indefinite
    lam.materials = [bad] + list(lam.materials[1:])
    for prec in (lib_mod.GL_PREC_FP64, lib_mod.GL_PREC_MIXED):
        with pytest.raises(lib_mod.GLError) as e:
            lib_mod.Solver.from_laminate(lam, precision=prec)
        assert e.value.code == -4      # GL_ERR_NOT_SPD


def test_out_of_device_memory_is_reported_and_recoverable(lib_mod):
    import torch
    lam = plate()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    hog = torch.empty(free - (16 << 20), dtype=torch.uint8, device="cuda")
    try:
        with pytest.raises(lib_mod.GLError) as e:
            lib_mod.Solver.from_laminate(lam)
        assert e.value.code == -2      # GL_ERR_OOM
    finally:
        del hog
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    s = lib_mod.Solver.from_laminate(lam)
    u, info = s.solve()
    assert info["status"] == 0 and info["rel_resid"] <= lam.tol

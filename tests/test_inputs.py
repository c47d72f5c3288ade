"""Input-description helpers (no GPU): the element masks that select the adjoint
objective's region and the misalignment patch agree with the oracle's own mesh
classification and with the stated geometry."""
import math

import numpy as np

from oracle import fem
from paper_1707_04228_gb300 import inputs


def test_resin_and_arc_masks_match_the_oracle_mesh():
    lam = inputs.corner_mini(n_arc=8, n_limb=2, n_width=6, nel_layer=2, angles=(0, 90), nsub=(4, 2, 1), nev=8,
                             width=6.0, wrinkle_w=1.0)
    mesh = fem.Mesh(lam)
    assert np.array_equal(inputs.resin_elements(lam), mesh.is_resin)
    tc = 0.5 * (lam.sv[mesh.eijk[:, 0]] + lam.sv[mesh.eijk[:, 0] + 1])
    assert np.array_equal(inputs.arc_resin_mask(lam), mesh.is_resin & (tc > 0) & (tc < 1))


def test_patch_mask_geometry_on_the_corner():
    lam = inputs.corner_c1()
    m = inputs.wrinkle_patch_mask(lam, 10.0, 10.0).reshape(lam.nz, lam.ny, lam.nx)
    s = inputs.centre_arc_length(lam)
    rmid = lam.R_inner + 0.5 * lam.thickness
    s0 = 0.5 * math.radians(lam.arc_deg) * rmid
    cols = np.flatnonzero(m.any(axis=(0, 1)))
    assert np.all(np.abs(s[cols] - s0) <= 5.0)
    lc = 0.5 * (lam.lv[:-1] + lam.lv[1:])
    rows = np.flatnonzero(m.any(axis=(0, 2)))
    assert np.all(np.abs(lc[rows] - 7.5) <= 5.0) and len(rows) == 20
    assert not np.any(m & inputs.resin_elements(lam).reshape(m.shape))
    # arc length is continuous across the limb/arc joints and grows monotonically
    assert np.all(np.diff(s) > 0)


def test_paper_corner_geometry():
    """The 39-ply corner: the printed stack (39 plies, 38 resin interfaces,
    T = 9.93 mm as the paper states), a wrinkle whose steepest fibre angle is
    about 10 degrees, and no folded node column."""
    lam = inputs.paper_corner()
    plies = [a for a, m in zip(lam.layer_angle_deg, lam.layer_mat) if m == 0]
    assert len(plies) == 39 and len(lam.layer_mat) == 77
    assert abs(lam.thickness - 9.93) < 1e-9
    assert sorted(set(plies)) == [-45.0, 0.0, 45.0, 90.0]
    assert 9.0 < np.degrees(np.abs(lam.theta).max()) < 11.0
    rn = inputs._q2_params(lam.rv())
    assert np.diff(rn[:, None, None] + lam.node_dr, axis=0).min() > 0
    assert lam.n_dof == 13_559_865


def test_paper_corner_edge_resin_strips():
    lam = inputs.paper_corner(n_arc=6, n_limb=1, n_width=4, edge_resin=3.0, n_edge=2, nsub=(2, 2, 1))
    assert np.allclose(lam.lv[[0, 2, -3, -1]], [-3.0, 0.0, 52.0, 55.0])
    em = lam.elem_mat
    assert em.shape == (lam.nz, lam.ny, lam.nx)
    assert np.all(em[:, :2, :] == 1) and np.all(em[:, -2:, :] == 1)
    inner = em[:, 2:-2, :]
    assert np.array_equal(inner[:, 0, 0], np.asarray(lam.layer_mat)[lam.elem_layer()])

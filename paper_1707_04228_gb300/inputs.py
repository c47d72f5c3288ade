"""Seeded synthetic laminate workloads (shared by the oracle and the CUDA path).

This module only *describes* inputs: 1D vertex coordinate arrays, the ply
stack, the material table, the per-element fibre-misalignment field and the
Dirichlet/traction data.  It contains none of the method's arithmetic (no
shape functions, no stiffness, no geometry map, no solver): the oracle and the
GPU library each build the mesh and the operator from this description on
their own.

Conventions (the library's boundary uses the same ones):
  * units N, mm, MPa;
  * structured Q2 mesh with nx x ny x nz elements; element e = ex + nx*(ey + ny*ez);
  * Q2 nodes (2nx+1) x (2ny+1) x (2nz+1), node n = ix + NX*(iy + NY*iz),
    x (the s / arc-length direction) fastest and z (thickness, r) slowest;
  * DOF = 3*node + component;
  * faces: 0 -s, 1 +s, 2 -l, 3 +l, 4 -r (inner/bottom), 5 +r (outer/top).

Materials follow the paper's Table 1 (Section 2.2): orthotropic ply
E11=162 GPa, E22=E33=10 GPa, G12=G13=5.2 GPa, G23=3.5 GPa, nu12=nu13=0.35,
nu23=0.5; isotropic resin interface E=10 GPa, nu=0.35.

The curved geometry is the corner-unfolding specimen of Section 2.2 and the
mapping of Section 3 (equation after eq-f): the s vertex array then holds a
parametric coordinate t with limb 1 on t in [-1,0], the arc on [0,1] and
limb 2 on [1,2] (the arc angle is arc_deg * t on [0,1]).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Table 1 (Section 2.2), MPa.
PLY_T1 = dict(kind="ortho", E1=162000.0, E2=10000.0, E3=10000.0,
              G12=5200.0, G13=5200.0, G23=3500.0,
              nu12=0.35, nu13=0.35, nu23=0.5)
RESIN_T1 = dict(kind="iso", E=10000.0, nu=0.35)

FACE_SM, FACE_SP, FACE_LM, FACE_LP, FACE_RM, FACE_RP = range(6)


@dataclass
class Laminate:
    """A layered hex laminate plus its loads and solver options."""
    name: str
    geometry: int                  # 0 flat, 1 curved
    sv: np.ndarray                 # s vertex coords (nx+1): mm (flat) or parametric t (curved)
    lv: np.ndarray                 # l (width) vertex coords (ny+1), mm
    layer_nel: list
    layer_thick: list              # mm
    layer_mat: list                # index into materials
    layer_angle_deg: list          # ply angle about the laminate normal
    materials: list                # dicts, see PLY_T1 / RESIN_T1
    R_inner: float = 0.0
    limb_L: float = 0.0
    arc_deg: float = 90.0
    theta: np.ndarray | None = None   # (nz, ny, nx) misalignment, rad
    node_dr: np.ndarray | None = None  # (NZ, NY, NX) through-thickness node offset (geometric wrinkle), mm
    elem_mat: np.ndarray | None = None  # (nz, ny, nx) material index overriding the layer's (edge resin strips)
    element: int = 0               # 0: 27-node Q2 hexahedra; 1: 20-node serendipity hexahedra (same node grid)
    periodic_width: int = 0        # 1: u equal on the width planes l = lv[0] and l = lv[-1]
    dir_dof: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    dir_val: np.ndarray = field(default_factory=lambda: np.zeros(0))
    traction: list = field(default_factory=list)   # [(face, (tx, ty, tz))] MPa, global axes
    px: int = 2
    py: int = 2
    pz: int = 2
    overlap: int = 1
    nev: int = 8
    tol: float = 1e-10

    @property
    def nx(self):
        return len(self.sv) - 1

    @property
    def ny(self):
        return len(self.lv) - 1

    @property
    def nz(self):
        return int(sum(self.layer_nel))

    @property
    def node_dims(self):
        return 2 * self.nx + 1, 2 * self.ny + 1, 2 * self.nz + 1

    @property
    def n_nodes(self):
        a, b, c = self.node_dims
        return a * b * c

    @property
    def n_dof(self):
        return 3 * self.n_nodes

    @property
    def n_elem(self):
        return self.nx * self.ny * self.nz

    @property
    def thickness(self):
        return float(sum(self.layer_thick))

    def rv(self):
        """Through-thickness vertex coordinates (nz+1), measured from the inner face."""
        out = [0.0]
        base = 0.0
        for n, h in zip(self.layer_nel, self.layer_thick):
            out.extend(base + h * (i + 1) / n for i in range(n))
            base += h
        return np.asarray(out)

    def elem_layer(self):
        """Layer index of each element row in z (nz,)."""
        return np.repeat(np.arange(len(self.layer_nel)), self.layer_nel)


def _nodes_from_vertices(v):
    """Parametric Q2 node coordinates: vertices at even, midpoints at odd indices."""
    v = np.asarray(v, dtype=np.float64)
    out = np.empty(2 * len(v) - 1)
    out[0::2] = v
    out[1::2] = 0.5 * (v[:-1] + v[1:])
    return out


def graded(n, a, b, ratio, fine_at_b=True):
    """n elements on [a, b], geometric sizes with largest/smallest = ratio."""
    if n == 1 or ratio == 1.0:
        return np.linspace(a, b, n + 1)
    q = ratio ** (1.0 / (n - 1))
    h = q ** np.arange(n)
    if fine_at_b:
        h = h[::-1]
    h = h / h.sum() * (b - a)
    v = np.concatenate([[a], a + np.cumsum(h)])
    v[-1] = b
    return v


def face_node_ids(lam: Laminate, face: int) -> np.ndarray:
    NX, NY, NZ = lam.node_dims
    ix, iy, iz = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    sel = {FACE_SM: ix == 0, FACE_SP: ix == NX - 1, FACE_LM: iy == 0,
           FACE_LP: iy == NY - 1, FACE_RM: iz == 0, FACE_RP: iz == NZ - 1}[face]
    nid = ix + NX * (iy + NY * iz)
    return np.sort(nid[sel].ravel())


def clamp_face(lam: Laminate, face: int, comps=(0, 1, 2)):
    nodes = face_node_ids(lam, face)
    dof = (3 * nodes[:, None] + np.asarray(comps)[None, :]).ravel()
    return dof.astype(np.int64), np.zeros(dof.size)


def merge_dirichlet(*pairs):
    d = {}
    for dof, val in pairs:
        for i, v in zip(np.asarray(dof).tolist(), np.asarray(val).tolist()):
            d[i] = v
    k = np.array(sorted(d), dtype=np.int64)
    return k, np.array([d[i] for i in k.tolist()])


def _stack_with_resin(angles, ply_t, resin_t, nel_ply, nel_resin):
    nel, th, mat, ang = [], [], [], []
    for i, a in enumerate(angles):
        if i > 0:
            nel.append(nel_resin); th.append(resin_t); mat.append(1); ang.append(0.0)
        nel.append(nel_ply); th.append(ply_t); mat.append(0); ang.append(float(a))
    return nel, th, mat, ang


def flat_plate_c0() -> Laminate:
    """20x20x2.06 mm [0/90]s plate, 8x8x14 Q2 elements, clamped at x=0, 1 MPa x-traction at x=20."""
    nel, th, mat, ang = _stack_with_resin([0, 90, 90, 0], 0.5, 0.02, 2, 2)
    lam = Laminate(name="flat_0_90s_8x8x14", geometry=0,
                   sv=np.linspace(0.0, 20.0, 9), lv=np.linspace(0.0, 20.0, 9),
                   layer_nel=nel, layer_thick=th, layer_mat=mat, layer_angle_deg=ang,
                   materials=[PLY_T1, RESIN_T1], px=2, py=2, pz=2, overlap=1, nev=8, tol=1e-10)
    lam.dir_dof, lam.dir_val = clamp_face(lam, FACE_SM)
    lam.traction = [(FACE_SP, (1.0, 0.0, 0.0))]
    return lam


def centre_arc_length(lam: Laminate):
    """Element-centre coordinate along the laminate (nx,): the arc length of the
    mid-thickness surface (curved; limbs included) or x (flat), in mm."""
    tc = 0.5 * (lam.sv[:-1] + lam.sv[1:])
    if lam.geometry != 1:
        return tc
    rmid = lam.R_inner + 0.5 * lam.thickness
    arc = math.radians(lam.arc_deg)
    return np.where(tc < 0, tc * lam.limb_L,
                    np.where(tc <= 1, tc * arc * rmid, arc * rmid + (tc - 1) * lam.limb_L))


def resin_elements(lam: Laminate):
    """Boolean per element (element order x fastest, then y, then z): isotropic resin
    (its layer's material, or its own where elem_mat overrides it)."""
    iso_of_mat = np.array([m["kind"] == "iso" for m in lam.materials])
    if lam.elem_mat is not None:
        return iso_of_mat[np.asarray(lam.elem_mat).reshape(-1)]
    ez = iso_of_mat[np.asarray(lam.layer_mat)][lam.elem_layer()]
    return np.broadcast_to(ez[:, None, None], (lam.nz, lam.ny, lam.nx)).reshape(-1).copy()


def arc_resin_mask(lam: Laminate):
    """Resin elements of the arc (centre parameter 0 < t < 1): the corner region whose
    through-thickness stress the adjoint objective aggregates."""
    tc = 0.5 * (lam.sv[:-1] + lam.sv[1:])
    arc = (tc > 0) & (tc < 1)
    return resin_elements(lam) & np.broadcast_to(arc[None, None, :], (lam.nz, lam.ny, lam.nx)).reshape(-1)


def wrinkle_patch_mask(lam: Laminate, size_s=10.0, size_l=10.0):
    """Ply (non-resin) elements whose centres lie in a size_s x size_l mm patch of
    the (s, l) surface centred mid-arc (mid-length when flat) and mid-width:
    the misalignment parameters of the adjoint study."""
    s = centre_arc_length(lam)
    if lam.geometry == 1:
        s0 = 0.5 * math.radians(lam.arc_deg) * (lam.R_inner + 0.5 * lam.thickness)
    else:
        s0 = 0.5 * (s[0] + s[-1])
    lc = 0.5 * (lam.lv[:-1] + lam.lv[1:])
    l0 = 0.5 * (lam.lv[0] + lam.lv[-1])
    ins = (np.abs(lc - l0)[:, None] <= 0.5 * size_l) & (np.abs(s - s0)[None, :] <= 0.5 * size_s)
    return ~resin_elements(lam) & np.broadcast_to(ins[None], (lam.nz, lam.ny, lam.nx)).reshape(-1)


def _q2_params(v):
    """Q2 node parameters of a vertex array: vertices and edge midpoints."""
    v = np.asarray(v, dtype=np.float64)
    out = np.empty(2 * len(v) - 1)
    out[0::2] = v
    out[1::2] = 0.5 * (v[:-1] + v[1:])
    return out


def sech2_wrinkle(lam: Laminate, d, b1=0.2, b2_inner=0.5, b2_outer=0.25, b3=0.5,
                  s_def=None, l_def=None, r_def=None, width=None):
    """The paper's geometric wrinkle (Section 3, Eqs. eq-wrinkle and eq-f):
    the through-thickness coordinate of every node moves by

        f = d sech^2(pi (s - s_def) / b1) sech^2(pi (r - r_def) / (T b2)) sech^2(pi (l - l_def) / (W b3)),

    b2 = b2_inner below r_def and b2_outer above it.  Readings: s is the arc
    parameter t on [0, 1] (the paper's s on [0, pi] divided by pi; for flat
    plates x divided by the length), r the depth from the inner face with the
    laminate thickness T as its scale (the printed "R b2"), W the width.  The
    fibres follow the wrinkled surfaces: theta_e = -atan(df/ds) at the element
    centre (s the arc length of the ply at that depth; R_l(theta) tilts e_s
    towards -r for theta > 0).  Returns (node_dr (NZ, NY, NX), theta (nz, ny, nx));
    defaults centre the defect mid-arc, mid-width and mid-thickness; width
    (default: the mesh's) is the part width W of the l factor."""
    T = lam.thickness
    W = float(lam.lv[-1] - lam.lv[0]) if width is None else float(width)
    sv = np.asarray(lam.sv, dtype=np.float64)
    if lam.geometry == 1:
        to_s = lambda t: t                                  # arc parameter
    else:
        S = float(sv[-1] - sv[0])
        to_s = lambda t: (t - sv[0]) / S
    s_def = 0.5 if s_def is None else s_def
    l_def = 0.5 * (lam.lv[0] + lam.lv[-1]) if l_def is None else l_def
    r_def = 0.5 * T if r_def is None else r_def

    def f_and_slope(t, l, r):
        a_s = math.pi * (to_s(t) - s_def) / b1
        b2 = np.where(r - r_def < 0, b2_inner, b2_outer)
        a_r = math.pi * (r - r_def) / (T * b2)
        a_l = math.pi * (l - l_def) / (W * b3)
        f = d / np.cosh(a_s) ** 2 / np.cosh(a_r) ** 2 / np.cosh(a_l) ** 2
        dfdu = -2.0 * np.tanh(a_s) * f * math.pi / b1       # d f / d(normalised s)
        if lam.geometry == 1:
            rr = lam.R_inner + r
            dsdt = np.where((t >= 0) & (t <= 1), rr * math.radians(lam.arc_deg), lam.limb_L)
            dfds = dfdu / dsdt
        else:
            dfds = dfdu / S
        return f, dfds

    tn, ln, rn = _q2_params(sv), _q2_params(lam.lv), _q2_params(lam.rv())
    Rg, Lg, Tg = np.meshgrid(rn, ln, tn, indexing="ij")   # (NZ, NY, NX)
    dr, _ = f_and_slope(Tg, Lg, Rg)
    tc = 0.5 * (sv[:-1] + sv[1:])
    lc = 0.5 * (lam.lv[:-1] + lam.lv[1:])
    rv = lam.rv()
    rc = 0.5 * (rv[:-1] + rv[1:])
    Rc, Lc, Tc = np.meshgrid(rc, lc, tc, indexing="ij")   # (nz, ny, nx)
    _, slope = f_and_slope(Tc, Lc, Rc)
    return dr, -np.arctan(slope)


def gaussian_theta(lam: Laminate, amp_deg, width_mm, s_centre=None, r_sigma=None,
                   l_centre=None, l_sigma=None):
    """Per-element misalignment theta(s, r) = A exp(-(s-s0)^2/2w^2) exp(-(r-r0)^2/2 sr^2).

    s is the arc length along the mid-thickness surface (curved) or x (flat),
    r the depth through the thickness; evaluated at parametric element centres.
    """
    T = lam.thickness
    rv = lam.rv()
    rc = 0.5 * (rv[:-1] + rv[1:])
    tc = 0.5 * (lam.sv[:-1] + lam.sv[1:])
    if lam.geometry == 1:
        rmid = lam.R_inner + 0.5 * T
        arc = math.radians(lam.arc_deg)
        s = np.where(tc < 0, tc * lam.limb_L,
                     np.where(tc <= 1, tc * arc * rmid, arc * rmid + (tc - 1) * lam.limb_L))
        s0 = 0.5 * arc * rmid if s_centre is None else s_centre
    else:
        s = tc
        s0 = 0.5 * (lam.sv[0] + lam.sv[-1]) if s_centre is None else s_centre
    sr = T / 4.0 if r_sigma is None else r_sigma
    gs = np.exp(-0.5 * ((s - s0) / width_mm) ** 2)
    gr = np.exp(-0.5 * ((rc - 0.5 * T) / sr) ** 2)
    th = math.radians(amp_deg) * gr[:, None, None] * np.ones((1, lam.ny, 1)) * gs[None, None, :]
    if l_sigma is not None:
        lc = 0.5 * (lam.lv[:-1] + lam.lv[1:])
        l0 = 0.5 * (lam.lv[0] + lam.lv[-1]) if l_centre is None else l_centre
        th = th * np.exp(-0.5 * ((lc - l0) / l_sigma) ** 2)[None, :, None]
    return th


def limb_end_rotation(lam: Laminate, delta):
    """Prescribed rigid rotation delta about the width axis of the limb-2 end face.

    The face is the +s face at the end of limb 2.  Its nodes sit at
    c + r e_r(psi_end) + l e_l, and a small rotation delta about e_l through the
    mid-thickness line gives u = delta (r - r_mid) d with d the limb direction.
    """
    NX, NY, NZ = lam.node_dims
    rn = lam.R_inner + _nodes_from_vertices(lam.rv())
    rmid = lam.R_inner + 0.5 * lam.thickness
    pe = math.radians(lam.arc_deg)
    d = np.array([math.cos(pe), 0.0, -math.sin(pe)])
    nodes = face_node_ids(lam, FACE_SP)
    iz = nodes // (NX * NY)
    u = delta * (rn[iz] - rmid)[:, None] * d[None, :]
    dof = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    return dof.astype(np.int64), u.ravel()


def curved_corner(n_arc=100, n_limb=10, n_width=30, nel_layer=4, width=15.0,
                  limb_L=50.0, R_inner=5.0, angles=(0, 90, 45, -45, 0, 90),
                  ply_t=0.25, resin_t=0.02, amp_deg=10.0, wrinkle_w=4.0,
                  delta=-1e-3, limb_bias=5.0, nsub=(16, 2, 4), nev=10, name=None) -> Laminate:
    """Curved corner-unfolding laminate (Section 2.2 / Section 3 geometry).

    Default: 90-degree arc of 5 mm inner radius with 50 mm limbs, 12 plies
    [0/90/+45/-45/0/90]s of 0.25 mm with 0.02 mm resin interfaces, 4 elements
    through each layer, 100 elements on the arc, 10 per limb (graded toward the
    arc), 30 across a 15 mm width: 120 x 30 x 92 elements.  Limb 1 is clamped,
    limb 2's end face gets a rigid opening rotation.
    """
    full = list(angles) + list(angles)[::-1]
    nel, th, mat, ang = _stack_with_resin(full, ply_t, resin_t, nel_layer, nel_layer)
    limb1 = graded(n_limb, -1.0, 0.0, limb_bias, fine_at_b=True) if n_limb else np.array([0.0])
    arc = np.linspace(0.0, 1.0, n_arc + 1)
    limb2 = graded(n_limb, 1.0, 2.0, limb_bias, fine_at_b=False) if n_limb else np.array([1.0])
    sv = np.concatenate([limb1[:-1], arc, limb2[1:]])
    lam = Laminate(name=name or f"curved_{len(sv)-1}x{n_width}x{sum(nel)}", geometry=1,
                   sv=sv, lv=np.linspace(0.0, width, n_width + 1),
                   layer_nel=nel, layer_thick=th, layer_mat=mat, layer_angle_deg=ang,
                   materials=[PLY_T1, RESIN_T1], R_inner=R_inner, limb_L=limb_L, arc_deg=90.0,
                   px=nsub[0], py=nsub[1], pz=nsub[2], overlap=1, nev=nev, tol=1e-10)
    if amp_deg:
        lam.theta = gaussian_theta(lam, amp_deg, wrinkle_w)
    lam.dir_dof, lam.dir_val = merge_dirichlet(clamp_face(lam, FACE_SM),
                                               limb_end_rotation(lam, delta))
    return lam


def corner_c1() -> Laminate:
    """The 8.16M-DOF curved corner: 120 x 30 x 92 Q2 elements, 128 subdomains, 10 eigenvectors."""
    return curved_corner(name="curved_corner_120x30x92")


# The 39-ply stacking sequence of the large corner study (Section 3):
# [[-+45/90/0]_2/[-+45]_2/90/-+45/90/0/-+45/0/+-45/0/90/+-45/90/[+-45]_2/[0/90/+-45]_2]
PAPER_39_PLY = ([-45, 45, 90, 0] * 2 + [-45, 45] * 2 + [90, -45, 45, 90, 0, -45, 45, 0, 45, -45, 0, 90, 45, -45, 90]
                + [45, -45] * 2 + [0, 90, 45, -45] * 2)


def paper_corner(n_arc=100, n_limb=10, n_width=60, d_wrinkle=0.62, delta=-1e-3, limb_bias=3.0,
                 nsub=(32, 4, 1), nev=10, edge_resin=0.0, n_edge=2, periodic=False, name=None) -> Laminate:
    """The geometry of the paper's 39-ply wrinkle study (Section 3): inner radius
    22 mm, 10 mm limbs, 52 mm width, 0.24 mm plies with 0.015 mm resin
    interfaces (T = 9.93 mm), the printed stacking sequence, one Q2 element
    through every ply and every interface (77 element layers), the sech^2
    geometric wrinkle of amplitude d_wrinkle mm centred mid-arc, mid-width and
    mid-thickness (0.62 mm gives a steepest fibre angle of about 10 degrees).
    Loads as for the other corners: limb 1 clamped, a rigid opening rotation
    of limb 2's end.  edge_resin > 0 adds the paper's resin strips of that
    width (mm, n_edge elements each) along both free edges of the width (all
    layers resin there); periodic=True applies the study's periodic width
    conditions instead (no free edges; one subdomain across the width, so
    nsub[1] is set to 1; the wrinkle is symmetric about mid-width, so the two
    width faces have the same shape).  Default mesh 120 x 60 x 77 elements,
    13,559,865 DOF."""
    assert len(PAPER_39_PLY) == 39
    nel, th, mat, ang = _stack_with_resin(PAPER_39_PLY, 0.24, 0.015, 1, 1)
    limb1 = graded(n_limb, -1.0, 0.0, limb_bias, fine_at_b=True) if n_limb else np.array([0.0])
    arc = np.linspace(0.0, 1.0, n_arc + 1)
    limb2 = graded(n_limb, 1.0, 2.0, limb_bias, fine_at_b=False) if n_limb else np.array([1.0])
    sv = np.concatenate([limb1[:-1], arc, limb2[1:]])
    lv = np.linspace(0.0, 52.0, n_width + 1)
    if edge_resin > 0:
        strip = np.linspace(0.0, edge_resin, n_edge + 1)
        lv = np.concatenate([strip[:-1] - edge_resin, lv, 52.0 + strip[1:]])
    lam = Laminate(name=name or f"paper_corner_{len(sv)-1}x{len(lv)-1}x{sum(nel)}", geometry=1,
                   sv=sv, lv=lv,
                   layer_nel=nel, layer_thick=th, layer_mat=mat, layer_angle_deg=ang,
                   materials=[PLY_T1, RESIN_T1], R_inner=22.0, limb_L=10.0, arc_deg=90.0,
                   px=nsub[0], py=nsub[1], pz=nsub[2], overlap=1, nev=nev, tol=1e-10)
    if edge_resin > 0:
        em = np.broadcast_to(np.asarray(mat)[lam.elem_layer()][:, None, None], (lam.nz, lam.ny, lam.nx)).copy()
        em[:, :n_edge, :] = 1
        em[:, -n_edge:, :] = 1
        lam.elem_mat = em
    if d_wrinkle:
        lam.node_dr, lam.theta = sech2_wrinkle(lam, d_wrinkle, width=52.0)
    lam.dir_dof, lam.dir_val = merge_dirichlet(clamp_face(lam, FACE_SM), limb_end_rotation(lam, delta))
    if periodic:
        assert edge_resin == 0, "periodic width conditions leave no free edge for resin strips"
        lam.periodic_width = 1
        lam.py = 1
    return lam


def corner_mini(n_arc=8, n_limb=0, n_width=6, nel_layer=2, angles=(0, 90), nsub=(2, 2, 2), nev=8,
                limb_L=5.0, width=6.0, amp_deg=10.0, wrinkle_w=1.0):
    """A small curved laminate of the same family, used for parity tests."""
    return curved_corner(n_arc=n_arc, n_limb=n_limb, n_width=n_width, nel_layer=nel_layer,
                         width=width, limb_L=limb_L, angles=angles, amp_deg=amp_deg,
                         wrinkle_w=wrinkle_w, nsub=nsub, nev=nev,
                         name=f"curved_mini_{n_arc + 2 * n_limb}x{n_width}")


def flat_random(rng: np.random.Generator, n_inplane, n_plies, amp_deg, nsub=(2, 2, 1), nev=6,
                ply_t=0.25, resin_t=0.02, size=20.0, name="flat_random"):
    """Flat plate with a random stack drawn from {0, +-45, 90}, 1 element per layer,
    a Gaussian misalignment patch of random centre and the C0 loads."""
    angles = rng.choice([0.0, 45.0, -45.0, 90.0], size=n_plies)
    nel, th, mat, ang = _stack_with_resin(angles, ply_t, resin_t, 1, 1)
    lam = Laminate(name=name, geometry=0, sv=np.linspace(0, size, n_inplane + 1),
                   lv=np.linspace(0, size, n_inplane + 1), layer_nel=nel, layer_thick=th,
                   layer_mat=mat, layer_angle_deg=ang, materials=[PLY_T1, RESIN_T1],
                   px=nsub[0], py=nsub[1], pz=nsub[2], overlap=1, nev=nev, tol=1e-10)
    if amp_deg > 0:
        lam.theta = gaussian_theta(lam, amp_deg, 4.0, s_centre=rng.uniform(0, size))
    lam.dir_dof, lam.dir_val = clamp_face(lam, FACE_SM)
    lam.traction = [(FACE_SP, (1.0, 0.0, 0.0))]
    return lam


def random_vector(n, seed):
    """Seeded standard-normal FP64 vector."""
    return np.random.default_rng(seed).standard_normal(n)


def batch_plates(count=96, seed=1707, dof_lo=40_000, dof_hi=800_000, nev=8):
    """Flat laminates of uneven sizes and stackings for the batched solve.

    Per laminate: a target size N ~ U[dof_lo, dof_hi]; a ply count P ~ U{4..24}
    with 0.25 mm plies and 0.02 mm resin between them, one element per layer
    (2P - 1 element layers); a square in-plane grid n x n, n in [10, 40],
    chosen so that 3 (2n+1)^2 (2(2P-1)+1) is nearest the target (P is redrawn
    until some n lands within 10%); ply angles iid from {0, +-45, 90}; a
    Gaussian misalignment patch of amplitude U[0, 12] degrees; clamped at x = 0
    with a 1 MPa x-traction at x = 20 mm.
    """
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        target = rng.uniform(dof_lo, dof_hi)
        pick = None
        for _ in range(200):
            P = int(rng.integers(4, 25))
            nz = 2 * P - 1
            n = int(round((math.sqrt(target / (3.0 * (2 * nz + 1))) - 1.0) / 2.0))
            if 10 <= n <= 40 and abs(3 * (2 * n + 1) ** 2 * (2 * nz + 1) - target) <= 0.1 * target:
                pick = (n, P)
                break
        if pick is None:
            continue
        amp = float(rng.uniform(0.0, 12.0))
        lam = flat_random(rng, pick[0], pick[1], amp, nsub=(0, 0, 1), nev=nev, name=f"plate_{len(out)}")
        out.append(lam)
    return out

"""ctypes binding of libgeneo_lam.so (C ABI in include/geneo_lam.h).

Argument marshalling only: every step of the solve runs inside the CUDA
library.  Arrays may be NumPy host arrays or CUDA torch tensors (their device
pointer is passed straight through).  There is no CPU fallback: if the
library cannot be loaded the import fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

_LIB_PATH = _build.LIB

GL_PREC_FP64, GL_PREC_MIXED = 0, 1
ERRORS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error", -4: "not SPD",
          -5: "not converged", -6: "NaN/Inf", -7: "timeout", -8: "call out of order"}


class GLError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)} ({code}): {msg}")
        self.code = code


class gl_ortho(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E1", "E2", "E3", "G12", "G13", "G23", "nu12", "nu13", "nu23")]


class gl_mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x", C.c_void_p), ("y", C.c_void_p),
                ("nlayers", C.c_int), ("layer_nel", C.c_void_p), ("layer_thick", C.c_void_p),
                ("layer_mat", C.c_void_p), ("layer_angle_deg", C.c_void_p), ("geometry", C.c_int),
                ("R_inner", C.c_double), ("limb_L", C.c_double), ("arc_deg", C.c_double),
                ("theta_e", C.c_void_p), ("node_dr", C.c_void_p), ("elem_mat", C.c_void_p), ("element", C.c_int),
                ("periodic_width", C.c_int)]


class gl_opts(C.Structure):
    _fields_ = [("px", C.c_int), ("py", C.c_int), ("pz", C.c_int), ("overlap", C.c_int), ("nev", C.c_int),
                ("max_iter", C.c_int), ("precision", C.c_int), ("resid_period", C.c_int),
                ("tol", C.c_double), ("sigma", C.c_double), ("eig_iters", C.c_int),
                ("factor_ws_bytes", C.c_double), ("eig_group_bytes", C.c_double), ("fp32_update", C.c_int),
                ("sweep_overlap", C.c_int)]


class gl_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("rel_resid", C.c_double),
                ("rel_resid_true", C.c_double), ("ms_setup", C.c_double), ("ms_solve", C.c_double),
                ("n_free", C.c_int64), ("n_coarse", C.c_int), ("factor_nnz", C.c_int64),
                ("n_coarse_dropped", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gl_profile_data(C.Structure):
    _fields_ = [("ms_ku", C.c_double), ("ms_local", C.c_double), ("ms_coarse", C.c_double),
                ("n_ku", C.c_int64), ("n_local", C.c_int64), ("n_coarse", C.c_int64),
                ("factor_entries", C.c_int64), ("local_dofs", C.c_int64), ("factor_bytes_per_entry", C.c_int),
                ("factor_levels", C.c_int), ("n_elem", C.c_int64), ("n_dof", C.c_int64), ("n_sub", C.c_int),
                ("n_coarse_dim", C.c_int), ("factor_nonzeros", C.c_int64), ("factor_groups", C.c_int),
                ("eig_groups", C.c_int), ("max_level_fronts", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# name -> (restype, argtypes)
SIGNATURES = {
    "gl_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "gl_destroy": (None, [C.c_void_p]),
    "gl_strerror": (C.c_char_p, [C.c_int]),
    "gl_last_error": (C.c_char_p, []),
    "gl_set_materials": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "gl_set_mesh": (C.c_int, [C.c_void_p, C.POINTER(gl_mesh)]),
    "gl_set_dirichlet": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "gl_set_traction": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "gl_setup": (C.c_int, [C.c_void_p, C.POINTER(gl_opts)]),
    "gl_num_dofs": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "gl_num_elems": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "gl_rhs": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gl_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(gl_info)]),
    "gl_solve_increment": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(gl_info)]),
    "gl_stress": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gl_stress_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gl_apply_K": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gl_apply_prec": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gl_geneo_eigenvalues": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "gl_failure_index": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_int64)]),
    "gl_set_theta": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gl_stress_vjp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gl_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(gl_info)]),
    "gl_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_void_p]),
    "gl_batch_setup": (C.c_int, [C.c_void_p, C.POINTER(gl_opts)]),
    "gl_batch_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gl_batch_grid": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gl_batch_destroy": (None, [C.c_void_p]),
    "gl_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "gl_profile_read": (C.c_int, [C.c_void_p, C.POINTER(gl_profile_data)]),
    "gl_profile_levels": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "gl_kernel_launches": (C.c_longlong, []),
    "gl_fp64_peak_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                     C.POINTER(C.c_double)]),
}

_lib = None


def load(path=None):
    """Load libgeneo_lam.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is not built; run paper_1707_04228_gb300._build.build() (needs nvcc)")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _ptr(a):
    """Device pointer of a CUDA tensor, or the data pointer of a contiguous NumPy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(a.ctypes.data)


def _check(lib, rc):
    if rc != 0:
        raise GLError(rc, lib.gl_last_error().decode())


def fp64_peak_probe(device=0, iters=4096, reps=20):
    """Measured FP64 FMA rate of the device (gl_fp64_peak_probe):
    returns (flops per second, SM count, timed milliseconds)."""
    lib = load()
    f, n, ms = C.c_double(), C.c_int(), C.c_double()
    _check(lib, lib.gl_fp64_peak_probe(device, iters, reps, C.byref(f), C.byref(n), C.byref(ms)))
    return f.value, n.value, ms.value


class Solver:
    """One laminate problem on one GPU: mesh + materials + loads -> setup -> solve/stress."""

    def __init__(self, device=0, stream=None):
        self.lib = load()
        self.ctx = C.c_void_p()
        sp = None
        if stream is not None:
            sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _check(self.lib, self.lib.gl_create(C.byref(self.ctx), device, sp))
        self._keep = []

    def close(self):
        if self.ctx:
            self.lib.gl_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ problem definition
    def set_materials(self, materials):
        ortho = [m for m in materials if m["kind"] == "ortho"]
        iso = [m for m in materials if m["kind"] == "iso"]
        if [m["kind"] for m in materials] != ["ortho"] * len(ortho) + ["iso"] * len(iso):
            raise ValueError("orthotropic materials must come before isotropic ones")
        arr = (gl_ortho * max(1, len(ortho)))()
        for i, m in enumerate(ortho):
            for k in ("E1", "E2", "E3", "G12", "G13", "G23", "nu12", "nu13", "nu23"):
                setattr(arr[i], k, m[k])
        en = np.array([[m["E"], m["nu"]] for m in iso], dtype=np.float64).reshape(-1)
        _check(self.lib, self.lib.gl_set_materials(self.ctx, len(ortho), C.cast(arr, C.c_void_p), len(iso),
                                                   _ptr(en) if en.size else None))

    def set_mesh(self, lam):
        x = np.ascontiguousarray(lam.sv, dtype=np.float64)
        y = np.ascontiguousarray(lam.lv, dtype=np.float64)
        nel = np.ascontiguousarray(lam.layer_nel, dtype=np.int32)
        th = np.ascontiguousarray(lam.layer_thick, dtype=np.float64)
        mat = np.ascontiguousarray(lam.layer_mat, dtype=np.int32)
        ang = np.ascontiguousarray(lam.layer_angle_deg, dtype=np.float64)
        theta = None if lam.theta is None else np.ascontiguousarray(np.asarray(lam.theta).reshape(-1), dtype=np.float64)
        dr = getattr(lam, "node_dr", None)
        dr = None if dr is None else np.ascontiguousarray(np.asarray(dr).reshape(-1), dtype=np.float64)
        em = getattr(lam, "elem_mat", None)
        em = None if em is None else np.ascontiguousarray(np.asarray(em).reshape(-1), dtype=np.int32)
        self._keep = [x, y, nel, th, mat, ang, theta, dr, em]
        m = gl_mesh(nx=len(x) - 1, ny=len(y) - 1, x=x.ctypes.data, y=y.ctypes.data, nlayers=len(nel),
                    layer_nel=nel.ctypes.data, layer_thick=th.ctypes.data, layer_mat=mat.ctypes.data,
                    layer_angle_deg=ang.ctypes.data, geometry=int(lam.geometry), R_inner=float(lam.R_inner),
                    limb_L=float(lam.limb_L), arc_deg=float(lam.arc_deg),
                    theta_e=None if theta is None else theta.ctypes.data,
                    node_dr=None if dr is None else dr.ctypes.data,
                    elem_mat=None if em is None else em.ctypes.data, element=int(getattr(lam, "element", 0)),
                    periodic_width=int(getattr(lam, "periodic_width", 0)))
        _check(self.lib, self.lib.gl_set_mesh(self.ctx, C.byref(m)))

    def set_dirichlet(self, dof, val):
        d = np.ascontiguousarray(dof, dtype=np.int64)
        v = np.ascontiguousarray(val, dtype=np.float64)
        _check(self.lib, self.lib.gl_set_dirichlet(self.ctx, d.size, _ptr(d), _ptr(v)))

    def set_traction(self, face, t):
        tv = np.ascontiguousarray(t, dtype=np.float64)
        _check(self.lib, self.lib.gl_set_traction(self.ctx, int(face), _ptr(tv)))

    def setup(self, px, py, pz, overlap=1, nev=8, tol=1e-10, max_iter=2000, precision=GL_PREC_FP64,
              resid_period=50, sigma=0.0, eig_iters=0, factor_ws_bytes=0.0, eig_group_bytes=0.0,
              fp32_update=0, sweep_overlap=0):
        o = gl_opts(px=px, py=py, pz=pz, overlap=overlap, nev=nev, max_iter=max_iter, precision=precision,
                    resid_period=resid_period, tol=tol, sigma=sigma, eig_iters=eig_iters,
                    factor_ws_bytes=factor_ws_bytes, eig_group_bytes=eig_group_bytes, fp32_update=fp32_update,
                    sweep_overlap=sweep_overlap)
        _check(self.lib, self.lib.gl_setup(self.ctx, C.byref(o)))

    @classmethod
    def from_laminate(cls, lam, device=0, stream=None, **opts):
        s = cls(device, stream)
        s.set_materials(lam.materials)
        s.set_mesh(lam)
        s.set_dirichlet(lam.dir_dof, lam.dir_val)
        for face, t in lam.traction:
            s.set_traction(face, t)
        kw = dict(px=lam.px, py=lam.py, pz=lam.pz, overlap=lam.overlap, nev=lam.nev, tol=lam.tol)
        kw.update(opts)
        s.setup(**kw)
        return s

    # ------------------------------------------------------------ queries / operations
    @property
    def n_dof(self):
        n = C.c_int64()
        _check(self.lib, self.lib.gl_num_dofs(self.ctx, C.byref(n)))
        return n.value

    @property
    def n_elem(self):
        n = C.c_int64()
        _check(self.lib, self.lib.gl_num_elems(self.ctx, C.byref(n)))
        return n.value

    def rhs(self, out=None):
        out = np.empty(self.n_dof) if out is None else out
        _check(self.lib, self.lib.gl_rhs(self.ctx, _ptr(out)))
        return out

    def solve(self, f=None, out=None, check=True):
        out = np.empty(self.n_dof) if out is None else out
        info = gl_info()
        rc = self.lib.gl_solve(self.ctx, _ptr(f), _ptr(out), C.byref(info))
        if check:
            _check(self.lib, rc)
        self.last_info = info.as_dict()
        return out, self.last_info

    def solve_increment(self, g, out=None, check=True):
        """gl_solve_increment: du with K_ff du_f = g_f and du = 0 on the Dirichlet DOFs."""
        out = np.empty(self.n_dof) if out is None else out
        info = gl_info()
        rc = self.lib.gl_solve_increment(self.ctx, _ptr(g), _ptr(out), C.byref(info))
        if check:
            _check(self.lib, rc)
        return out, info.as_dict()

    def stress(self, u, s33=None, t13=None):
        ne = self.n_elem
        s33 = np.empty(ne) if s33 is None else s33
        t13 = np.empty(ne) if t13 is None else t13
        peak = np.zeros(1)
        _check(self.lib, self.lib.gl_stress(self.ctx, _ptr(u), _ptr(s33), _ptr(t13), _ptr(peak)))
        return s33, t13, float(peak[0])

    def stress_noalloc(self, u, s33, t13, peak=None):
        """gl_stress_noalloc: u, s33, t13 and peak (or None) are caller-owned
        device buffers (torch tensors or raw device addresses); nothing is
        allocated and the call returns before the work on the context's stream
        is done."""
        def dptr(a, n, name):
            if a is None or isinstance(a, int):
                return None if a is None else C.c_void_p(a)
            if hasattr(a, "data_ptr"):
                import torch
                if a.dtype != torch.float64 or not a.is_cuda or a.numel() < n:
                    raise ValueError(f"{name}: needs a CUDA float64 tensor of at least {n} entries")
            return _ptr(a)
        ne = self.n_elem
        _check(self.lib, self.lib.gl_stress_noalloc(self.ctx, dptr(u, self.n_dof, "u"), dptr(s33, ne, "s33"),
                                                    dptr(t13, ne, "t13"), dptr(peak, 1, "peak")))

    def apply_K(self, x, out=None):
        out = np.empty(self.n_dof) if out is None else out
        _check(self.lib, self.lib.gl_apply_K(self.ctx, _ptr(x), _ptr(out)))
        return out

    def apply_prec(self, r, out=None):
        out = np.empty(self.n_dof) if out is None else out
        _check(self.lib, self.lib.gl_apply_prec(self.ctx, _ptr(r), _ptr(out)))
        return out

    def failure_index(self, u, s33=61.0, s13=97.0, F=None):
        """Quadratic damage-onset criterion per element; returns (F, peak, peak element)."""
        F = np.empty(self.n_elem) if F is None else F
        peak = np.zeros(1)
        elem = C.c_int64()
        _check(self.lib, self.lib.gl_failure_index(self.ctx, _ptr(u), s33, s13, _ptr(F), _ptr(peak), C.byref(elem)))
        return F, float(peak[0]), elem.value

    def set_theta(self, theta):
        t = theta if hasattr(theta, "data_ptr") else np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
        _check(self.lib, self.lib.gl_set_theta(self.ctx, _ptr(t)))

    def stress_vjp(self, u, w33=None, w13=None, dJdu=None, dJdtheta=None, want_u=True, want_theta=True):
        if want_u and dJdu is None:
            dJdu = np.empty(self.n_dof)
        if want_theta and dJdtheta is None:
            dJdtheta = np.empty(self.n_elem)
        _check(self.lib, self.lib.gl_stress_vjp(self.ctx, _ptr(u), _ptr(w33), _ptr(w13), _ptr(dJdu),
                                                _ptr(dJdtheta)))
        return dJdu, dJdtheta

    def adjoint(self, u, dJdu, grad=None):
        grad = np.empty(self.n_elem) if grad is None else grad
        info = gl_info()
        _check(self.lib, self.lib.gl_adjoint(self.ctx, _ptr(u), _ptr(dJdu), _ptr(grad), C.byref(info)))
        self.last_adjoint_info = info.as_dict()
        return grad, self.last_adjoint_info

    def profile(self, enable=True):
        """gl_profile: True or 1 times the solve's phases, 2 also every dissection level of the
        local solves (levels then in sequence), False or 0 switches timing off."""
        mode = 1 if enable is True else (0 if enable is False else int(enable))
        _check(self.lib, self.lib.gl_profile(self.ctx, mode))

    def profile_read(self):
        d = gl_profile_data()
        _check(self.lib, self.lib.gl_profile_read(self.ctx, C.byref(d)))
        return d.as_dict()

    def profile_levels(self):
        """gl_profile_levels: per dissection level, the timed forward/backward sweep milliseconds,
        fronts, factor nonzeros, padded block entries and largest front, plus the number of timed
        applications."""
        n, calls = C.c_int(), C.c_int64()
        _check(self.lib, self.lib.gl_profile_levels(self.ctx, 0, None, None, None, None, None, None, C.byref(n),
                                                    C.byref(calls)))
        L = n.value
        fwd, bwd = np.zeros(L), np.zeros(L)
        fronts, nz, pad = (np.zeros(L, dtype=np.int64) for _ in range(3))
        maxf = np.zeros(L, dtype=np.int32)
        _check(self.lib, self.lib.gl_profile_levels(self.ctx, L, _ptr(fwd), _ptr(bwd), _ptr(fronts), _ptr(nz),
                                                    _ptr(pad), _ptr(maxf), C.byref(n), C.byref(calls)))
        return {"calls": calls.value, "fwd_ms": fwd, "bwd_ms": bwd, "fronts": fronts, "nonzeros": nz,
                "padded": pad, "max_front": maxf}

    def kernel_launches(self):
        return int(self.lib.gl_kernel_launches())

    def geneo_eigenvalues(self):
        n = C.c_int()
        _check(self.lib, self.lib.gl_geneo_eigenvalues(self.ctx, None, 0, C.byref(n)))
        out = np.empty(n.value)
        if n.value:
            _check(self.lib, self.lib.gl_geneo_eigenvalues(self.ctx, _ptr(out), n.value, C.byref(n)))
        return out


class Batch:
    """Many laminates solved together (gl_batch_*): one launch per phase for all of them,
    one PCG iteration replayed as a CUDA graph."""

    def __init__(self, laminates, device=0, stream=None):
        self.lib = load()
        self.solvers = []
        for lam in laminates:
            s = Solver(device, None)
            s.set_materials(lam.materials)
            s.set_mesh(lam)
            s.set_dirichlet(lam.dir_dof, lam.dir_val)
            for face, t in lam.traction:
                s.set_traction(face, t)
            self.solvers.append(s)
        arr = (C.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        self.b = C.c_void_p()
        sp = None
        if stream is not None:
            sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _check(self.lib, self.lib.gl_batch_create(C.byref(self.b), len(self.solvers), C.cast(arr, C.c_void_p), sp))

    def setup(self, px=0, py=0, overlap=1, nev=8, tol=1e-10, max_iter=2000, precision=GL_PREC_FP64,
              resid_period=50, sigma=0.0, eig_iters=0, factor_ws_bytes=0.0, eig_group_bytes=0.0,
              fp32_update=0):
        o = gl_opts(px=px, py=py, pz=1, overlap=overlap, nev=nev, max_iter=max_iter, precision=precision,
                    resid_period=resid_period, tol=tol, sigma=sigma, eig_iters=eig_iters,
                    factor_ws_bytes=factor_ws_bytes, eig_group_bytes=eig_group_bytes, fp32_update=fp32_update)
        _check(self.lib, self.lib.gl_batch_setup(self.b, C.byref(o)))

    def grid(self):
        out = np.zeros(2 * len(self.solvers), dtype=np.int32)
        _check(self.lib, self.lib.gl_batch_grid(self.b, _ptr(out)))
        return out.reshape(-1, 2)

    def solve(self, outs=None, check=True):
        n = len(self.solvers)
        if outs is None:
            outs = [np.empty(s.n_dof) for s in self.solvers]
        ptrs = (C.c_void_p * n)(*[_ptr(o).value for o in outs])
        infos = (gl_info * n)()
        rc = self.lib.gl_batch_solve(self.b, C.cast(ptrs, C.c_void_p), C.cast(infos, C.c_void_p))
        if check:
            _check(self.lib, rc)
        return outs, [infos[i].as_dict() for i in range(n)]

    def close(self):
        if self.b:
            self.lib.gl_batch_destroy(self.b)
            self.b = C.c_void_p()
        for s in self.solvers:
            s.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

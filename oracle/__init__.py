"""FP64 CPU oracle of the BA-/AB-GMRES reconstruction path (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package; the CUDA library and its
Python binding never import it.  It shares no code with them.

* ``ct_oracle.c`` (plain C, FP64, OpenMP): the projector A (Joseph), the
  voxel-driven back-projector B_un, the ramp filter F and the exact
  transposes, Sec. I Eq. 1 and Sec. III of the paper.
* ``krylov.py`` (numpy, FP64): BA-GMRES (Eq. 5), AB-GMRES (Eq. 4) and
  CGLS (Eqs. 2-3) on top of any operator pair.
* ``analytic.py``: closed-form line integrals of ellipsoids, used to pin A.

Every function here is pinned by the ``-m "not gpu"`` tests
(tests/test_oracle_*.py); nothing is "parity unpinned" except what the
module docstrings of those tests say.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ct_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libctoracle.so")


def build(force: bool = False) -> str:
    """Compile ct_oracle.c with gcc (OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Geom(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("vox", ctypes.c_double), ("n_views", ctypes.c_int),
                ("ang0", ctypes.c_double), ("span", ctypes.c_double), ("nu", ctypes.c_int),
                ("nv", ctypes.c_int), ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("sod", ctypes.c_double), ("sdd", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, L = ctypes.c_double, ctypes.c_long
        g = P(_Geom)
        sig = {
            "or_project_A": [g, P(d), P(d)],
            "or_project_A_rays": [g, P(d), P(L), L, P(d)],
            "or_adjoint_At": [g, P(d), P(d)],
            "or_backproject_B": [g, P(d), P(d)],
            "or_backproject_B_voxels": [g, P(d), P(L), L, P(d)],
            "or_adjoint_Bt": [g, P(d), P(d)],
            "or_ramp_F": [g, P(d), P(d)],
            "or_ramp_Ft": [g, P(d), P(d)],
            "or_ramp_F_rows": [g, P(d), P(L), L, P(d)],
            "or_project_S": [g, P(d), P(d)],
            "or_project_S_rays": [g, P(d), P(L), L, P(d)],
            "or_adjoint_St": [g, P(d), P(d)],
            "or_s_row": [g, L, P(L), P(d)],
            "or_s_row_capacity": [g],
            "or_a_row": [g, L, P(L), P(d)],
            "or_b_row": [g, L, P(L), P(d)],
            "or_a_row_capacity": [g],
            "or_b_row_capacity": [g],
            "or_ramp_scale": [g],
            "or_num_threads": [],
        }
        for name, args in sig.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = None
        for name in ("or_a_row", "or_b_row", "or_s_row", "or_a_row_capacity", "or_b_row_capacity",
                     "or_s_row_capacity", "or_num_threads"):
            getattr(_lib, name).restype = ctypes.c_int
        _lib.or_ramp_scale.restype = ctypes.c_double
    return _lib


def _geom(g) -> _Geom:
    return _Geom(g.kind, g.nx, g.ny, g.nz, g.vox, g.n_views, g.ang0, g.span, g.nu, g.nv,
                 g.du, g.dv, g.sod, g.sdd)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _f64(a, size):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if a.size != size:
        raise ValueError("expected %d elements, got %d" % (size, a.size))
    return a


def num_threads() -> int:
    return lib().or_num_threads()


# --- operators (Sec. I Eq. 1; Sec. III) -----------------------------------------
def project_A(g, x):
    """y = A x (Joseph ray-driven projector), shape (n_views, nv, nu)."""
    x = _f64(x, g.n)
    y = np.empty(g.m)
    lib().or_project_A(ctypes.byref(_geom(g)), _dptr(x), _dptr(y))
    return y.reshape(g.sino_shape)


def project_A_rays(g, x, rays):
    """(A x)[rays] for flat ray indices (view*nv + v)*nu + u."""
    x = _f64(x, g.n)
    rays = np.ascontiguousarray(rays, dtype=np.int64)
    out = np.empty(rays.size)
    lib().or_project_A_rays(ctypes.byref(_geom(g)), _dptr(x), _lptr(rays), rays.size, _dptr(out))
    return out


def project_S(g, x):
    """y = A_S x (line-intersection projector: ray length inside each voxel)."""
    x = _f64(x, g.n)
    y = np.empty(g.m)
    lib().or_project_S(ctypes.byref(_geom(g)), _dptr(x), _dptr(y))
    return y.reshape(g.sino_shape)


def project_S_rays(g, x, rays):
    """(A_S x)[rays] for flat ray indices."""
    x = _f64(x, g.n)
    rays = np.ascontiguousarray(rays, dtype=np.int64)
    out = np.empty(rays.size)
    lib().or_project_S_rays(ctypes.byref(_geom(g)), _dptr(x), _lptr(rays), rays.size, _dptr(out))
    return out


def adjoint_St(g, y):
    """x = A_S^T y (exact transpose of A_S)."""
    y = _f64(y, g.m)
    x = np.empty(g.n)
    lib().or_adjoint_St(ctypes.byref(_geom(g)), _dptr(y), _dptr(x))
    return x.reshape(g.vol_shape)


def s_row(g, ray):
    """(voxel indices, lengths) of row `ray` of A_S."""
    cap = lib().or_s_row_capacity(ctypes.byref(_geom(g)))
    idx = np.empty(cap, dtype=np.int64)
    w = np.empty(cap)
    cnt = lib().or_s_row(ctypes.byref(_geom(g)), int(ray), _lptr(idx), _dptr(w))
    return idx[:cnt].copy(), w[:cnt].copy()


def adjoint_At(g, y):
    """x = A^T y (exact transpose of A)."""
    y = _f64(y, g.m)
    x = np.empty(g.n)
    lib().or_adjoint_At(ctypes.byref(_geom(g)), _dptr(y), _dptr(x))
    return x.reshape(g.vol_shape)


def ramp_F(g, y):
    """F y: cosine weight + Ram-Lak row convolution (B_FBP = B_un F)."""
    y = _f64(y, g.m)
    out = np.empty(g.m)
    lib().or_ramp_F(ctypes.byref(_geom(g)), _dptr(y), _dptr(out))
    return out.reshape(g.sino_shape)


def ramp_Ft(g, z):
    """F^T z."""
    z = _f64(z, g.m)
    out = np.empty(g.m)
    lib().or_ramp_Ft(ctypes.byref(_geom(g)), _dptr(z), _dptr(out))
    return out.reshape(g.sino_shape)


def ramp_F_rows(g, y, rows):
    """Rows (flat index view*nv + v) of F y, shape (len(rows), nu)."""
    y = _f64(y, g.m)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.size * g.nu)
    lib().or_ramp_F_rows(ctypes.byref(_geom(g)), _dptr(y), _lptr(rows), rows.size, _dptr(out))
    return out.reshape(rows.size, g.nu)


def ramp_scale(g) -> float:
    return lib().or_ramp_scale(ctypes.byref(_geom(g)))


def backproject_B(g, y, filtered=False):
    """x = B y with B = B_un (voxel-driven) or B_FBP = B_un F."""
    y = _f64(y, g.m)
    if filtered:
        y = ramp_F(g, y).reshape(-1)
    x = np.empty(g.n)
    lib().or_backproject_B(ctypes.byref(_geom(g)), _dptr(y), _dptr(x))
    return x.reshape(g.vol_shape)


def backproject_B_voxels(g, y, voxels, filtered=False):
    """(B y)[voxels] for flat voxel indices."""
    y = _f64(y, g.m)
    if filtered:
        y = ramp_F(g, y).reshape(-1)
    voxels = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty(voxels.size)
    lib().or_backproject_B_voxels(ctypes.byref(_geom(g)), _dptr(y), _lptr(voxels), voxels.size,
                                  _dptr(out))
    return out


def adjoint_Bt(g, x, filtered=False):
    """y = B^T x: B_un^T, or B_FBP^T = F^T B_un^T."""
    x = _f64(x, g.n)
    y = np.empty(g.m)
    lib().or_adjoint_Bt(ctypes.byref(_geom(g)), _dptr(x), _dptr(y))
    if filtered:
        y = ramp_Ft(g, y).reshape(-1)
    return y.reshape(g.sino_shape)


def a_row(g, ray):
    """(voxel indices, weights) of row `ray` of A."""
    cap = lib().or_a_row_capacity(ctypes.byref(_geom(g)))
    idx = np.empty(cap, dtype=np.int64)
    w = np.empty(cap)
    cnt = lib().or_a_row(ctypes.byref(_geom(g)), int(ray), _lptr(idx), _dptr(w))
    return idx[:cnt].copy(), w[:cnt].copy()


def b_row(g, voxel):
    """(sinogram indices, weights) of row `voxel` of B_un."""
    cap = lib().or_b_row_capacity(ctypes.byref(_geom(g)))
    idx = np.empty(cap, dtype=np.int64)
    w = np.empty(cap)
    cnt = lib().or_b_row(ctypes.byref(_geom(g)), int(voxel), _lptr(idx), _dptr(w))
    return idx[:cnt].copy(), w[:cnt].copy()


class Operators:
    """The pair (A, B) of one geometry as flat-vector callables for the solvers;
    projector "joseph" (A) or "siddon" (A_S)."""

    def __init__(self, g, b_kind="un", projector="joseph"):
        self.g = g
        self.b_kind = b_kind
        self.siddon = projector == "siddon"

    def A(self, x):
        return (project_S if self.siddon else project_A)(self.g, x).reshape(-1)

    def B(self, y):
        if self.b_kind in ("At", "at"):
            return (adjoint_St if self.siddon else adjoint_At)(self.g, y).reshape(-1)
        return backproject_B(self.g, y, filtered=self.b_kind == "fbp").reshape(-1)


class AdjointOperators:
    """A^T and B^T of one geometry as flat-vector callables."""

    def __init__(self, g, b_kind="un"):
        self.g = g
        self.b_kind = b_kind

    def At(self, y):
        return adjoint_At(self.g, y).reshape(-1)

    def Bt(self, x):
        return adjoint_Bt(self.g, x, filtered=self.b_kind == "fbp").reshape(-1)


from . import krylov, analytic  # noqa: E402,F401

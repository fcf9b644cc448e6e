"""ctypes binding of libct (include/ct.h).

Argument marshalling only: every step of the reconstruction runs in the CUDA
library.  Tensors are torch CUDA tensors (float32, contiguous) on the
geometry's device; the stream is torch's current stream unless given.  There
is no CPU fallback: when libct.so is missing the import fails with a message
saying how to build it.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# CT_LIB=checked selects the index-checked build (libct_checked.so, see
# ct_bounds_checked in include/ct.h); the default is the regular build
LIB_PATH = os.path.join(_HERE, "_build", "libct_checked.so" if os.environ.get("CT_LIB") == "checked"
                        else "libct.so")

CT_OK, CT_EINVAL, CT_ENOMEM, CT_ECUDA, CT_ENONFINITE, CT_ETIMEOUT, CT_BREAKDOWN_LUCKY = range(7)
CT_PARALLEL_2D, CT_CONE_3D = 0, 1
CT_F32, CT_BF16 = 0, 1
CT_PROJ_JOSEPH, CT_PROJ_SIDDON = 0, 1
PROJECTORS = {"joseph": CT_PROJ_JOSEPH, "siddon": CT_PROJ_SIDDON}
CT_B_UN, CT_B_FBP, CT_B_AT = 0, 1, 2
CT_SOLVER_BA, CT_SOLVER_AB, CT_SOLVER_CGLS, CT_SOLVER_BA_VJP = 0, 1, 2, 3

B_KINDS = {"un": CT_B_UN, "fbp": CT_B_FBP, "at": CT_B_AT, "At": CT_B_AT}

STATUS_NAMES = {0: "CT_OK", 1: "CT_EINVAL", 2: "CT_ENOMEM", 3: "CT_ECUDA", 4: "CT_ENONFINITE",
                5: "CT_ETIMEOUT", 6: "CT_BREAKDOWN_LUCKY"}


class ct_geom_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("voxel_mm", ctypes.c_double), ("n_views", ctypes.c_int),
                ("angle_start_rad", ctypes.c_double), ("angle_span_rad", ctypes.c_double),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int), ("du_mm", ctypes.c_double),
                ("dv_mm", ctypes.c_double), ("sod_mm", ctypes.c_double), ("sdd_mm", ctypes.c_double),
                ("vol_dtype", ctypes.c_int), ("sino_dtype", ctypes.c_int), ("projector", ctypes.c_int)]


class ct_solve_opts(ctypes.Structure):
    _fields_ = [("b_kind", ctypes.c_int), ("tol", ctypes.c_double), ("dot_mode", ctypes.c_int),
                ("reorth", ctypes.c_int), ("record_data_resid", ctypes.c_int),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


# name -> (restype, argtypes), mirroring include/ct.h
_P, _vp, _i, _sz, _d = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
SIGNATURES = {
    "ct_solve_opts_default": (None, [_P(ct_solve_opts)]),
    "ct_geom_create": (_i, [_P(ct_geom_desc), _P(_vp)]),
    "ct_geom_destroy": (None, [_vp]),
    "ct_geom_n": (_sz, [_vp]),
    "ct_geom_m": (_sz, [_vp]),
    "ct_project_A": (_i, [_vp, _vp, _vp, _vp]),
    "ct_backproject_B": (_i, [_vp, _vp, _vp, _i, _vp]),
    "ct_project_A_noalloc": (_i, [_vp, _vp, _vp, _vp]),
    "ct_adjoint_At": (_i, [_vp, _vp, _vp, _vp]),
    "ct_adjoint_Bt": (_i, [_vp, _vp, _vp, _i, _vp]),
    "ct_ramp_F": (_i, [_vp, _vp, _vp, _i, _vp]),
    "ct_bagmres_solve": (_i, [_vp, _vp, _i, _vp, _P(_d), _P(ct_solve_opts), _P(_i), _vp]),
    "ct_bagmres_solve_host": (_i, [_vp, _vp, _i, _vp, _P(_d), _P(ct_solve_opts), _P(_i), _vp]),
    "ct_bagmres_solve_err": (_i, [_vp, _vp, _i, _vp, _vp, _P(_d), _P(_d), _P(ct_solve_opts), _P(_i), _vp]),
    "ct_bagmres_restarted": (_i, [_vp, _vp, _i, _i, _vp, _P(_d), _P(ct_solve_opts), _P(_i), _vp]),
    "ct_abgmres_solve": (_i, [_vp, _vp, _i, _vp, _P(_d), _P(ct_solve_opts), _P(_i), _vp]),
    "ct_cgls_solve": (_i, [_vp, _vp, _i, _vp, _P(_d), _P(ct_solve_opts), _P(_i), _vp]),
    "ct_bagmres_vjp": (_i, [_vp, _vp, _i, _vp, _P(_d), _P(ct_solve_opts), _P(_i), _vp]),
    "ct_workspace_bytes": (_sz, [_vp, _i, _i, _P(ct_solve_opts)]),
    "ct_mgs_sweep": (_i, [_vp, _sz, _i, _sz, _vp, _vp, _i, _vp]),
    "ct_basis_combine": (_i, [_vp, _sz, _i, _sz, _vp, _vp, _vp]),
    "ct_profile_enable": (None, [_i]),
    "ct_profile_reset": (None, []),
    "ct_profile_read": (_i, [_P(_d), _P(ctypes.c_longlong), _i]),
    "ct_profile_kind_name": (ctypes.c_char_p, [_i]),
    "ct_measure_gather_peak": (_i, [_i, _P(_d), _vp]),
    "ct_bagmres_state_create": (_i, [_vp, _i, _i, _P(ct_solve_opts), _P(_vp)]),
    "ct_bagmres_state_start": (_i, [_vp, _vp, _vp]),
    "ct_bagmres_state_extend": (_i, [_vp, _i, _vp, _P(_d), _P(_i), _vp]),
    "ct_gmres_state_iters": (_i, [_vp]),
    "ct_gmres_state_basis_bytes": (_sz, [_vp, _i]),
    "ct_gmres_state_save": (_i, [_vp, ctypes.c_char_p, _vp]),
    "ct_gmres_state_load": (_i, [_vp, ctypes.c_char_p, _i, _i, _P(_vp), _vp]),
    "ct_gmres_state_destroy": (None, [_vp]),
    "ct_fault_set": (_i, [ctypes.c_char_p]),
    "ct_fault_get": (ctypes.c_char_p, []),
    "ct_bounds_checked": (_i, []),
    "ct_bounds_take": (_i, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_ulonglong)]),
    "ct_last_error": (ctypes.c_char_p, []),
    "ct_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libct (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built: run `python -c \"import __graft_entry__ as g; "
                               "g.build()\"` or `python paper_2201_07408_gb300/build.py`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class CTError(RuntimeError):
    """A C-ABI call returned an error status.  For a solver, ``result`` holds
    what the call reported before it stopped (iterations done and the residual
    history, -1 after the last iteration done), else None."""

    def __init__(self, name, status, result=None):
        self.status = status
        self.result = result
        msg = lib().ct_last_error().decode(errors="replace")
        super().__init__("%s failed with %s: %s" % (name, STATUS_NAMES.get(status, status), msg))


def _check(name, status, allow=(CT_OK,), result=None):
    if status not in allow:
        raise CTError(name, status, result)
    return status


def _stream(stream, device):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t: torch.Tensor, numel: int, name: str, device) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float32:
        raise TypeError("%s must be float32 (got %s)" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    if t.device != device:
        raise ValueError("%s is on %s, the geometry on %s" % (name, t.device, device))
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t: torch.Tensor, numel: int, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
        raise TypeError("%s must be a CPU tensor" % name)
    if t.dtype != torch.float32:
        raise TypeError("%s must be float32 (got %s)" % (name, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


class Geometry:
    """A ct_geom handle (scan description uploaded to one CUDA device).

    Fields follow ct_geom_desc; ``from_spec`` accepts any object with the
    attributes kind, nx, ny, nz, vox, n_views, ang0, span, nu, nv, du, dv,
    sod, sdd.  ``projector``: "joseph" (default) or "siddon"."""

    def __init__(self, kind, nx, ny, nz, vox, n_views, ang0, span, nu, nv, du, dv, sod=0.0, sdd=0.0,
                 device=None, vol_dtype=CT_F32, sino_dtype=CT_F32, projector="joseph"):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.desc = ct_geom_desc(int(kind), int(nx), int(ny), int(nz), float(vox), int(n_views), float(ang0),
                                 float(span), int(nu), int(nv), float(du), float(dv), float(sod), float(sdd),
                                 _dtype(vol_dtype), _dtype(sino_dtype),
                                 PROJECTORS[projector] if isinstance(projector, str) else int(projector))
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check("ct_geom_create", lib().ct_geom_create(ctypes.byref(self.desc), ctypes.byref(self._h)))
        self.n = int(lib().ct_geom_n(self._h))
        self.m = int(lib().ct_geom_m(self._h))
        self.vol_shape = (int(nz), int(ny), int(nx))
        self.sino_shape = (int(n_views), int(nv), int(nu))

    @classmethod
    def from_spec(cls, spec, device=None, vol_dtype=CT_F32, sino_dtype=CT_F32, projector="joseph"):
        return cls(spec.kind, spec.nx, spec.ny, spec.nz, spec.vox, spec.n_views, spec.ang0, spec.span,
                   spec.nu, spec.nv, spec.du, spec.dv, spec.sod, spec.sdd, device=device,
                   vol_dtype=vol_dtype, sino_dtype=sino_dtype, projector=projector)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().ct_geom_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dtype(d) -> int:
    if isinstance(d, str):
        return {"f32": CT_F32, "fp32": CT_F32, "bf16": CT_BF16}[d]
    if d is torch.bfloat16:
        return CT_BF16
    if d is torch.float32:
        return CT_F32
    return int(d)


def _bkind(b_kind) -> int:
    if isinstance(b_kind, str):
        return B_KINDS[b_kind]
    return int(b_kind)


# --- C-ABI mirrors ----------------------------------------------------------------
def ct_project_A(geom: Geometry, x, y, stream=None):
    d = geom.device
    _check("ct_project_A", lib().ct_project_A(geom.handle, _ptr(x, geom.n, "x", d), _ptr(y, geom.m, "y", d),
                                              _stream(stream, d)))


def ct_project_A_noalloc(geom: Geometry, x, y, stream=None):
    """y = A x without any device allocation (fixed 32 MiB library scratch);
    see ct_project_A_noalloc in include/ct.h for the limit and sharing rules."""
    d = geom.device
    _check("ct_project_A_noalloc", lib().ct_project_A_noalloc(geom.handle, _ptr(x, geom.n, "x", d),
                                                              _ptr(y, geom.m, "y", d), _stream(stream, d)))


def ct_backproject_B(geom: Geometry, y, x, b_kind=CT_B_UN, stream=None):
    d = geom.device
    _check("ct_backproject_B", lib().ct_backproject_B(geom.handle, _ptr(y, geom.m, "y", d),
                                                      _ptr(x, geom.n, "x", d), _bkind(b_kind), _stream(stream, d)))


def ct_adjoint_At(geom: Geometry, y, x, stream=None):
    d = geom.device
    _check("ct_adjoint_At", lib().ct_adjoint_At(geom.handle, _ptr(y, geom.m, "y", d), _ptr(x, geom.n, "x", d),
                                                _stream(stream, d)))


def ct_adjoint_Bt(geom: Geometry, x, y, b_kind=CT_B_UN, stream=None):
    d = geom.device
    _check("ct_adjoint_Bt", lib().ct_adjoint_Bt(geom.handle, _ptr(x, geom.n, "x", d), _ptr(y, geom.m, "y", d),
                                                _bkind(b_kind), _stream(stream, d)))


def ct_ramp_F(geom: Geometry, y, yf, transpose=False, stream=None):
    d = geom.device
    _check("ct_ramp_F", lib().ct_ramp_F(geom.handle, _ptr(y, geom.m, "y", d), _ptr(yf, geom.m, "yf", d),
                                        int(bool(transpose)), _stream(stream, d)))


def make_opts(b_kind=CT_B_UN, tol=0.0, dot_mode=0, reorth=0, record_data_resid=False, workspace=None):
    o = ct_solve_opts()
    lib().ct_solve_opts_default(ctypes.byref(o))
    o.b_kind = _bkind(b_kind)
    o.tol = float(tol)
    o.dot_mode = int(dot_mode)
    o.reorth = int(reorth)
    o.record_data_resid = int(bool(record_data_resid))
    if workspace is not None:
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def ct_workspace_bytes(geom: Geometry, k: int, solver: int, opts: Optional[ct_solve_opts] = None) -> int:
    return int(lib().ct_workspace_bytes(geom.handle, int(k), int(solver),
                                        ctypes.byref(opts) if opts is not None else None))


@dataclass
class SolveResult:
    status: int
    iters: int
    resid: np.ndarray   # (k+1,) FP64, -1 after the last iteration done


def _solve(name, fn, solver, geom, b, k, x_out, opts, stream, workspace):
    d = geom.device
    if opts is None:
        opts = make_opts()
    if workspace == "torch":
        nbytes = ct_workspace_bytes(geom, k, solver, opts)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=d)
        opts.workspace = ctypes.c_void_p(ws.data_ptr())
        opts.workspace_bytes = nbytes
    resid = np.zeros(int(k) + 1, dtype=np.float64)
    iters = ctypes.c_int(0)
    st = fn(geom.handle, _ptr(b, geom.m, "b", d), int(k), _ptr(x_out, geom.n, "x_out", d),
            resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts), ctypes.byref(iters),
            _stream(stream, d))
    out = SolveResult(status=st, iters=iters.value, resid=resid)
    _check(name, st, allow=(CT_OK, CT_BREAKDOWN_LUCKY), result=out)
    return out


def ct_bagmres_solve(geom, b, k, x_out, opts=None, stream=None, workspace="torch") -> SolveResult:
    """BA-GMRES, k iterations on B A x = B b (Eq. 5); x_out receives x_k."""
    return _solve("ct_bagmres_solve", lib().ct_bagmres_solve, CT_SOLVER_BA, geom, b, k, x_out, opts, stream,
                  workspace)


def ct_bagmres_solve_host(geom, b_host, k, x_out_host, opts=None, stream=None, workspace="torch") -> SolveResult:
    """BA-GMRES with b and x_k in host memory (CPU float32 tensors; pinned
    ones give asynchronous copies): copy in, solve, copy out, in one call."""
    d = geom.device
    if opts is None:
        opts = make_opts()
    if workspace == "torch":
        nbytes = ct_workspace_bytes(geom, k, CT_SOLVER_BA, opts)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=d)
        opts.workspace = ctypes.c_void_p(ws.data_ptr())
        opts.workspace_bytes = nbytes
    resid = np.zeros(int(k) + 1, dtype=np.float64)
    iters = ctypes.c_int(0)
    st = lib().ct_bagmres_solve_host(geom.handle, _host_ptr(b_host, geom.m, "b_host"), int(k),
                                     _host_ptr(x_out_host, geom.n, "x_out_host"),
                                     resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts),
                                     ctypes.byref(iters), _stream(stream, d))
    out = SolveResult(status=st, iters=iters.value, resid=resid)
    _check("ct_bagmres_solve_host", st, allow=(CT_OK, CT_BREAKDOWN_LUCKY), result=out)
    return out


def _torch_workspace(geom, k, solver, opts):
    nbytes = ct_workspace_bytes(geom, k, solver, opts)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=geom.device)
    opts.workspace = ctypes.c_void_p(ws.data_ptr())
    opts.workspace_bytes = nbytes
    return ws


def ct_bagmres_solve_err(geom, b, k, x_out, x_ref, opts=None, stream=None, workspace="torch"):
    """BA-GMRES with the image error of every iterate: returns
    (SolveResult, err) with err[j] = ||x_j - x_ref|| (numpy, k+1; -1 after
    the last iteration done)."""
    d = geom.device
    if opts is None:
        opts = make_opts()
    ws = _torch_workspace(geom, k, CT_SOLVER_BA, opts) if workspace == "torch" else None
    resid = np.zeros(int(k) + 1, dtype=np.float64)
    err = np.zeros(int(k) + 1, dtype=np.float64)
    iters = ctypes.c_int(0)
    st = lib().ct_bagmres_solve_err(geom.handle, _ptr(b, geom.m, "b", d), int(k), _ptr(x_out, geom.n, "x_out", d),
                                    _ptr(x_ref, geom.n, "x_ref", d),
                                    resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    err.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts),
                                    ctypes.byref(iters), _stream(stream, d))
    del ws
    _check("ct_bagmres_solve_err", st, allow=(CT_OK, CT_BREAKDOWN_LUCKY))
    return SolveResult(status=st, iters=iters.value, resid=resid), err


def ct_bagmres_restarted(geom, b, m, cycles, x_out, opts=None, stream=None, workspace="torch") -> SolveResult:
    """Restarted BA-GMRES(m): `cycles` cycles of m iterations, each on the
    residual system; resid has m*cycles + 1 entries."""
    d = geom.device
    if opts is None:
        opts = make_opts()
    ws = _torch_workspace(geom, m, CT_SOLVER_BA, opts) if workspace == "torch" else None
    resid = np.zeros(int(m) * int(cycles) + 1, dtype=np.float64)
    iters = ctypes.c_int(0)
    st = lib().ct_bagmres_restarted(geom.handle, _ptr(b, geom.m, "b", d), int(m), int(cycles),
                                    _ptr(x_out, geom.n, "x_out", d),
                                    resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts),
                                    ctypes.byref(iters), _stream(stream, d))
    del ws
    _check("ct_bagmres_restarted", st, allow=(CT_OK, CT_BREAKDOWN_LUCKY))
    return SolveResult(status=st, iters=iters.value, resid=resid)


def ct_abgmres_solve(geom, b, k, x_out, opts=None, stream=None, workspace="torch") -> SolveResult:
    """AB-GMRES, k iterations on A B y = b, x = B y (Eq. 4)."""
    return _solve("ct_abgmres_solve", lib().ct_abgmres_solve, CT_SOLVER_AB, geom, b, k, x_out, opts, stream,
                  workspace)


def ct_cgls_solve(geom, b, k, x_out, opts=None, stream=None, workspace="torch") -> SolveResult:
    """CGLS with back-projector opts.b_kind in place of A^T (Eqs. 2-3)."""
    return _solve("ct_cgls_solve", lib().ct_cgls_solve, CT_SOLVER_CGLS, geom, b, k, x_out, opts, stream,
                  workspace)


def ct_bagmres_vjp(geom, gx, k, gb_out, opts=None, stream=None, workspace="torch") -> SolveResult:
    """dL/db = B^T (A^T B^T)^{-1} gx through a converged BA-GMRES solve
    (k GMRES iterations on A^T B^T); gb_out (m floats) receives it."""
    d = geom.device
    if opts is None:
        opts = make_opts()
    if workspace == "torch":
        nbytes = ct_workspace_bytes(geom, k, CT_SOLVER_BA_VJP, opts)
        ws = torch.empty(nbytes, dtype=torch.uint8, device=d)
        opts.workspace = ctypes.c_void_p(ws.data_ptr())
        opts.workspace_bytes = nbytes
    resid = np.zeros(int(k) + 1, dtype=np.float64)
    iters = ctypes.c_int(0)
    st = lib().ct_bagmres_vjp(geom.handle, _ptr(gx, geom.n, "gx", d), int(k), _ptr(gb_out, geom.m, "gb", d),
                              resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts),
                              ctypes.byref(iters), _stream(stream, d))
    out = SolveResult(status=st, iters=iters.value, resid=resid)
    _check("ct_bagmres_vjp", st, allow=(CT_OK, CT_BREAKDOWN_LUCKY), result=out)
    return out


CT_BASIS_DEVICE, CT_BASIS_HOST = 0, 1


class GmresState:
    """A persistent BA-GMRES solve (ct_bagmres_state_*): start(b), then
    extend(k) as often as wanted; save(path) / GmresState.load(...)."""

    def __init__(self, geom: "Geometry", kmax: int, basis="device", opts=None, _handle=None):
        self.geom = geom
        self.kmax = int(kmax)
        self.basis = CT_BASIS_HOST if basis in ("host", CT_BASIS_HOST) else CT_BASIS_DEVICE
        if _handle is not None:
            self._h = _handle
            return
        h = ctypes.c_void_p()
        _check("ct_bagmres_state_create",
               lib().ct_bagmres_state_create(geom.handle, self.kmax, self.basis,
                                             ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
        self._h = h

    @classmethod
    def load(cls, geom, path, kmax, basis="device", stream=None):
        h = ctypes.c_void_p()
        b = CT_BASIS_HOST if basis in ("host", CT_BASIS_HOST) else CT_BASIS_DEVICE
        _check("ct_gmres_state_load", lib().ct_gmres_state_load(geom.handle, str(path).encode(), int(kmax), b,
                                                                 ctypes.byref(h), _stream(stream, geom.device)))
        return cls(geom, kmax, b, _handle=h)

    def start(self, b, stream=None):
        d = self.geom.device
        _check("ct_bagmres_state_start", lib().ct_bagmres_state_start(self._h, _ptr(b, self.geom.m, "b", d),
                                                                      _stream(stream, d)))

    def extend(self, k, x_out, stream=None) -> SolveResult:
        d = self.geom.device
        resid = np.zeros(int(k) + 1, dtype=np.float64)
        iters = ctypes.c_int(0)
        st = lib().ct_bagmres_state_extend(self._h, int(k), _ptr(x_out, self.geom.n, "x_out", d),
                                           resid.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.byref(iters), _stream(stream, d))
        out = SolveResult(status=st, iters=iters.value, resid=resid)
        _check("ct_bagmres_state_extend", st, allow=(CT_OK, CT_BREAKDOWN_LUCKY), result=out)
        return out

    @property
    def iters(self) -> int:
        return int(lib().ct_gmres_state_iters(self._h))

    def save(self, path, stream=None):
        _check("ct_gmres_state_save", lib().ct_gmres_state_save(self._h, str(path).encode(),
                                                                _stream(stream, self.geom.device)))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ct_gmres_state_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ct_mgs_sweep(V, ldv, j, length, q, h, dot_mode=0, stream=None):
    """One MGS sweep of q against j basis vectors stored with stride ldv in V;
    h (float64 CUDA tensor of j+1) receives the coefficients and ||q||."""
    if h.dtype != torch.float64 or not h.is_cuda or h.numel() < j + 1:
        raise ValueError("h must be a float64 CUDA tensor of at least j+1 elements")
    d = q.device
    vptr = ctypes.c_void_p(V.data_ptr()) if V is not None else None
    _check("ct_mgs_sweep", lib().ct_mgs_sweep(vptr, int(ldv), int(j), int(length), _ptr(q, length, "q", d),
                                              ctypes.c_void_p(h.data_ptr()), int(dot_mode), _stream(stream, d)))


def ct_basis_combine(V, ldv, k, length, y, x, stream=None):
    """x = sum_{i<k} y[i] V_i (y float64 CUDA tensor)."""
    if y.dtype != torch.float64 or not y.is_cuda or y.numel() < k:
        raise ValueError("y must be a float64 CUDA tensor of at least k elements")
    d = x.device
    _check("ct_basis_combine", lib().ct_basis_combine(ctypes.c_void_p(V.data_ptr()), int(ldv), int(k),
                                                      int(length), ctypes.c_void_p(y.data_ptr()),
                                                      _ptr(x, length, "x", d), _stream(stream, d)))


def profile_enable(on=True):
    """Per-kernel CUDA-event timing inside the library (ct_profile_enable)."""
    lib().ct_profile_enable(int(bool(on)))


def profile_reset():
    lib().ct_profile_reset()


def profile_read():
    """{kernel kind: (device ms, launches)} accumulated since profile_reset()."""
    n = 32
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    k = lib().ct_profile_read(ms, cnt, n)
    return {lib().ct_profile_kind_name(i).decode(): (ms[i], int(cnt[i])) for i in range(min(k, n))}


def measure_gather_peak(repeats=5, stream=None, device=None):
    """GB/s of the SM load path's ceiling (ct_measure_gather_peak)."""
    d = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    out = ctypes.c_double(0.0)
    _check("ct_measure_gather_peak", lib().ct_measure_gather_peak(int(repeats), ctypes.byref(out),
                                                                  _stream(stream, d)))
    return out.value


def fault_set(spec):
    """Sets the host-side fault injection (ct_fault_set): "nan_at_iter:N",
    "oom", a comma-separated list, or None / "" / "none" to clear."""
    _check("ct_fault_set", lib().ct_fault_set(None if spec is None else spec.encode()))


def fault_get() -> str:
    return lib().ct_fault_get().decode()


BOUNDS_SITES = {1: "A z rows", 2: "A row window", 3: "A^T row window", 4: "B row", 5: "B column",
                6: "Siddon voxel offset"}


def bounds_checked() -> bool:
    """True when the loaded library is the index-checked build."""
    return bool(lib().ct_bounds_checked())


def decode_bounds_record(rec: int):
    """(site, view or slice, value) of a ct_bounds_take record, None for 0."""
    if not rec:
        return None
    site = rec >> 56
    where = (rec >> 32) & 0xFFFFFF
    value = rec & 0xFFFFFFFF
    if value >= 1 << 31:
        value -= 1 << 32
    return site, where, value


def bounds_take(g):
    """Takes and clears the geometry's first failed index check (checked
    builds): None, or (site, view or slice, value) as decode_bounds_record."""
    rec = ctypes.c_ulonglong(0)
    _check("ct_bounds_take", lib().ct_bounds_take(g.handle, ctypes.byref(rec)))
    return decode_bounds_record(int(rec.value))


def version() -> str:
    return lib().ct_version().decode()


# --- conveniences ------------------------------------------------------------------
def project_A(geom, x, stream=None):
    y = torch.empty(geom.sino_shape, dtype=torch.float32, device=geom.device)
    ct_project_A(geom, x.contiguous(), y, stream)
    return y


def backproject_B(geom, y, b_kind="un", stream=None):
    x = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    ct_backproject_B(geom, y.contiguous(), x, b_kind, stream)
    return x


def adjoint_At(geom, y, stream=None):
    x = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    ct_adjoint_At(geom, y.contiguous(), x, stream)
    return x


def adjoint_Bt(geom, x, b_kind="un", stream=None):
    y = torch.empty(geom.sino_shape, dtype=torch.float32, device=geom.device)
    ct_adjoint_Bt(geom, x.contiguous(), y, b_kind, stream)
    return y


def ramp_F(geom, y, transpose=False, stream=None):
    out = torch.empty(geom.sino_shape, dtype=torch.float32, device=geom.device)
    ct_ramp_F(geom, y.contiguous(), out, transpose, stream)
    return out


def bagmres(geom, b, k, b_kind="un", tol=0.0, dot_mode=0, reorth=0, stream=None):
    x = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    res = ct_bagmres_solve(geom, b.contiguous(), k, x,
                           make_opts(b_kind=b_kind, tol=tol, dot_mode=dot_mode, reorth=reorth), stream)
    return x, res


def abgmres(geom, b, k, b_kind="un", tol=0.0, dot_mode=0, reorth=0, stream=None):
    x = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    res = ct_abgmres_solve(geom, b.contiguous(), k, x,
                           make_opts(b_kind=b_kind, tol=tol, dot_mode=dot_mode, reorth=reorth), stream)
    return x, res


def cgls(geom, b, k, b_kind="un", tol=0.0, record_data_resid=False, stream=None):
    x = torch.empty(geom.vol_shape, dtype=torch.float32, device=geom.device)
    res = ct_cgls_solve(geom, b.contiguous(), k, x,
                        make_opts(b_kind=b_kind, tol=tol, record_data_resid=record_data_resid), stream)
    return x, res

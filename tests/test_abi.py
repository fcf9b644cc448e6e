"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; argument validation that happens before any CUDA call works
without a GPU.  No compute call is made here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"CT_API[^;(]*?\b(ct_\w+)\s*\(", text, flags=re.S))
    return names


@pytest.fixture(scope="module")
def libct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_07408_gb300 import ct
    return ct


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("ct_geom_create", "ct_project_A", "ct_backproject_B", "ct_adjoint_At",
                     "ct_bagmres_solve", "ct_abgmres_solve", "ct_cgls_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libct):
    L = ctypes.CDLL(libct.LIB_PATH)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libct):
    assert declared_symbols() == set(libct.SIGNATURES)


def test_version_and_defaults(libct):
    assert "sm_103a" in libct.version()
    o = libct.ct_solve_opts()
    libct.lib().ct_solve_opts_default(ctypes.byref(o))
    assert o.b_kind == libct.CT_B_UN and o.dot_mode == 0 and o.reorth == 0 and o.tol == 0.0
    assert not o.workspace


def _desc(libct, **kw):
    base = dict(kind=1, nx=16, ny=16, nz=16, voxel_mm=1.0, n_views=8, angle_start_rad=0.0,
                angle_span_rad=6.283185307179586, nu=24, nv=16, du_mm=1.5, dv_mm=1.5, sod_mm=500.0,
                sdd_mm=1000.0, vol_dtype=0, sino_dtype=0)
    base.update(kw)
    return libct.ct_geom_desc(**base)


@pytest.mark.parametrize("bad", [dict(nx=0), dict(n_views=-1), dict(voxel_mm=0.0), dict(kind=7),
                                 dict(kind=0, nz=4), dict(kind=0, nz=1, nv=3), dict(sdd_mm=400.0),
                                 dict(nx=2000, ny=2000, voxel_mm=1.0), dict(vol_dtype=5), dict(sino_dtype=7),
                                 dict(du_mm=-1.0), dict(angle_span_rad=float("nan"))])
def test_geometry_validation_rejects_bad_descriptions(libct, bad):
    h = ctypes.c_void_p()
    d = _desc(libct, **bad)
    st = libct.lib().ct_geom_create(ctypes.byref(d), ctypes.byref(h))
    assert st == libct.CT_EINVAL
    assert not h.value
    assert libct.lib().ct_last_error()


def test_null_arguments_are_rejected(libct):
    L = libct.lib()
    assert L.ct_geom_create(None, None) == libct.CT_EINVAL
    assert L.ct_project_A(None, None, None, None) == libct.CT_EINVAL
    assert L.ct_bagmres_solve(None, None, 5, None, None, None, None, None) == libct.CT_EINVAL
    assert L.ct_workspace_bytes(None, 5, 0, None) == 0
    L.ct_geom_destroy(None)


@pytest.mark.parametrize("spec,canon", [("nan_at_iter:5", "nan_at_iter:5"), ("oom", "oom"),
                                        ("oom,nan_at_iter:12", "nan_at_iter:12,oom"), ("none", ""), ("", "")])
def test_fault_spec_parsing(libct, spec, canon):
    L = libct.lib()
    assert L.ct_fault_set(spec.encode()) == libct.CT_OK
    assert L.ct_fault_get().decode() == canon
    assert L.ct_fault_set(None) == libct.CT_OK and L.ct_fault_get() == b""


@pytest.mark.parametrize("bad", ["nan_at_iter:0", "nan_at_iter:", "nan_at_iter:x", "nan_at_iter:3x", "segv",
                                 "oom,,bogus"])
def test_fault_spec_rejects_malformed(libct, bad):
    L = libct.lib()
    assert L.ct_fault_set(b"oom") == libct.CT_OK
    assert L.ct_fault_set(bad.encode()) == libct.CT_EINVAL
    assert b"ct_fault_set" in L.ct_last_error()
    assert L.ct_fault_get() == b"oom"          # unchanged
    L.ct_fault_set(None)


@pytest.mark.parametrize("env,canon,warns", [("nan_at_iter:7", "nan_at_iter:7", False), ("bogus", "", True)])
def test_fault_spec_from_environment(libct, env, canon, warns):
    import subprocess
    import sys
    code = ("import ctypes; L = ctypes.CDLL(%r); L.ct_fault_get.restype = ctypes.c_char_p; "
            "print(L.ct_fault_get().decode())" % libct.LIB_PATH)
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, CT_FAULT=env), capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == canon
    assert ("ignoring CT_FAULT" in r.stderr) == warns


def test_checked_build_exports_every_declared_symbol_and_reports_itself(libct):
    from paper_2201_07408_gb300 import build
    Lc = ctypes.CDLL(build.LIB_CHECKED)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(Lc, n)]
    assert not missing, missing
    assert Lc.ct_bounds_checked() == 1
    assert ctypes.CDLL(build.LIB).ct_bounds_checked() == 0


def test_bounds_take_rejects_null_arguments(libct):
    L = libct.lib()
    rec = ctypes.c_ulonglong(7)
    assert L.ct_bounds_take(None, ctypes.byref(rec)) == libct.CT_EINVAL
    assert b"ct_bounds_take" in L.ct_last_error()


@pytest.mark.parametrize("site,where,value", [(4, 17, -3), (1, 359, 12), (6, 0, 2**31 - 1), (2, 2**24 - 1, -2**31)])
def test_bounds_record_decoding(libct, site, where, value):
    rec = (site << 56) | (where << 32) | (value & 0xFFFFFFFF)
    assert libct.decode_bounds_record(rec) == (site, where, value)
    assert libct.decode_bounds_record(0) is None

"""Runs the library's operators and solvers through the index-checked build
(libct_checked.so, CT_LIB=checked) and prints one JSON line with the bounds
record each call left on its geometry.  Called by tests/test_gpu_checked.py
in a child process, so that the checked library is the only one loaded.

    python tests/checked_run.py all       every operator and solver on the small and degenerate scans
    python tests/checked_run.py random    every operator on the seeded random scans
    python tests/checked_run.py margin    B_un on cone_small (run with CT_DEBUG_PADV set)
    python tests/checked_run.py zsafe     A on a tall-detector scan (run with CT_DEBUG_A_ZSAFE set)

Records are (site, view or slice, value) as ct.decode_bounds_record, or
null.  Nothing here reads outside a buffer: a failed check redirects the
access into range before it is made.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import ct_inputs as ci  # noqa: E402
from paper_2201_07408_gb300 import ct  # noqa: E402

# a scan whose detector rows reach far above and below the 8-slice volume:
# the projector's z rows leave the zero border, so it must clamp (a_zsafe 0)
TALL = ci._cone("tall_detector", 0, 2.0, 30, 48, 40, 3.0, nxyz=(32, 32, 8))
RANDOM_SCANS = 24   # ct_inputs.random_geometry(0..23)


def operators(g, spec, out):
    x = torch.from_numpy(ci.phantom(spec)[0]).cuda()
    y = ct.project_A(g, x)
    out.append(("A", ct.bounds_take(g)))
    for kind in ("un", "fbp"):
        ct.backproject_B(g, y, kind)
        out.append(("B_" + kind, ct.bounds_take(g)))
        ct.adjoint_Bt(g, x, kind)
        out.append(("Bt_" + kind, ct.bounds_take(g)))
    ct.adjoint_At(g, y)
    out.append(("At", ct.bounds_take(g)))
    ct.ramp_F(g, y)
    ct.ramp_F(g, y, transpose=True)
    out.append(("F", ct.bounds_take(g)))
    return y


def solvers(g, spec, y, out):
    for kind in ("un", "fbp"):
        ct.bagmres(g, y, 6, b_kind=kind)
        out.append(("ba_" + kind, ct.bounds_take(g)))
    ct.abgmres(g, y, 6)
    out.append(("ab", ct.bounds_take(g)))
    ct.cgls(g, y, 6, record_data_resid=True)
    out.append(("cgls", ct.bounds_take(g)))
    x = torch.empty(spec.vol_shape, device="cuda")
    ct.ct_bagmres_restarted(g, y, 3, 2, x)
    out.append(("restarted", ct.bounds_take(g)))
    gb = torch.empty(spec.sino_shape, device="cuda")
    gx = torch.from_numpy(ci.smooth_volume(spec, seed=3).astype(np.float32).reshape(spec.vol_shape)).cuda()
    ct.ct_bagmres_vjp(g, gx, 4, gb)
    out.append(("vjp", ct.bounds_take(g)))


def run_all():
    res = {}
    specs = [ci.CONE_SMALL, ci.CONE_ANISO, ci.CONE_THIN, ci.CONE_Z40, ci.PAR2D_ANISO, TALL] + ci.DEGENERATE
    for spec in specs:
        for storage, projector in (("f32", "joseph"), ("bf16", "joseph"), ("f32", "siddon")):
            if projector == "siddon" and spec.kind != ci.CONE_3D:
                continue
            out = []
            g = ct.Geometry.from_spec(spec, vol_dtype=storage, sino_dtype=storage, projector=projector)
            y = operators(g, spec, out)
            if storage == "f32":
                solvers(g, spec, y, out)
            g.close()
            res["%s/%s/%s" % (spec.name, storage, projector)] = out
    return res


def run_random(count):
    """Every operator (FP32, BF16, line intersection) on seeded random scans."""
    res = {}
    for seed in range(count):
        spec = ci.random_geometry(seed)
        for storage, projector in (("f32", "joseph"), ("bf16", "joseph"), ("f32", "siddon")):
            if projector == "siddon" and spec.kind != ci.CONE_3D:
                continue
            out = []
            g = ct.Geometry.from_spec(spec, vol_dtype=storage, sino_dtype=storage, projector=projector)
            y = operators(g, spec, out)
            if storage == "f32" and projector == "joseph":
                ct.bagmres(g, y, 4, b_kind="fbp")
                out.append(("ba_fbp", ct.bounds_take(g)))
            g.close()
            res["%s/%s/%s" % (spec.name, storage, projector)] = out
    return res


def run_one(spec, what):
    g = ct.Geometry.from_spec(spec)
    x = torch.from_numpy(ci.phantom(spec)[0]).cuda()
    y = ct.project_A(g, x)
    res = {"A": ct.bounds_take(g)}
    if what == "margin":
        ct.backproject_B(g, y, "un")
        res["B_un"] = ct.bounds_take(g)
    return res


def main():
    mode = sys.argv[1]
    assert ct.bounds_checked(), "CT_LIB=checked must select libct_checked.so"
    if mode == "all":
        res = run_all()
    elif mode == "margin":
        res = run_one(ci.CONE_SMALL, "margin")
    elif mode == "random":
        res = run_random(int(sys.argv[2]) if len(sys.argv) > 2 else RANDOM_SCANS)
    elif mode == "zsafe":
        res = run_one(TALL, "zsafe")
    else:
        raise SystemExit("unknown mode %s" % mode)
    torch.cuda.synchronize()
    print(json.dumps(res))


if __name__ == "__main__":
    main()

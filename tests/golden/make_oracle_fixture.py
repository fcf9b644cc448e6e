"""Writes oracle_tiny_cases.json: outputs of the FP64 oracle (and of nothing
else) on two tiny seeded scans, a 2D parallel-beam one (8 x 8 pixels, 12
views over 180 degrees, 13 bins) and a cone-beam one (8^3 voxels of 10 mm,
12 views, 13 x 9 detector of 14 mm, start angle 0.2 rad).

Stored per scan: A x for a seeded positive x (Sec. III, the projector),
B_un y and B_FBP y for a seeded y (Sec. III, the back-projectors), and the
BA-GMRES residual history ||B(b - A x_j)|| and final iterate for k = 8 on
b = A x (Eq. 5, x0 = 0), with B = B_un and B = B_FBP.

Run from the repository root:  python tests/golden/make_oracle_fixture.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ct_inputs as ci  # noqa: E402
import oracle  # noqa: E402
from oracle import krylov  # noqa: E402

K = 8
CASES = {
    "tiny2d": ci.Geometry("tiny2d", ci.PARALLEL_2D, 8, 8, 1, 1.0, 12, 0.0, math.pi, 13, 1, 1.0, 1.0),
    "tinycone": ci._cone("tinycone", 8, 10.0, 12, 13, 9, 14.0, ang0=0.2),
}


def spec_dict(g):
    return {k: getattr(g, k) for k in ("kind", "nx", "ny", "nz", "vox", "n_views", "ang0", "span", "nu", "nv",
                                        "du", "dv", "sod", "sdd")}


def case_outputs(g):
    x = ci.random_vector(g.n, 11, positive=True)
    y = ci.random_vector(g.m, 12, positive=True)
    out = {"spec": spec_dict(g), "x_seed": 11, "y_seed": 12, "k": K,
           "Ax": oracle.project_A(g, x).reshape(-1).tolist(),
           "Bun_y": oracle.backproject_B(g, y).reshape(-1).tolist(),
           "Bfbp_y": oracle.backproject_B(g, y, filtered=True).reshape(-1).tolist()}
    b = oracle.project_A(g, x).reshape(-1)
    for kind in ("un", "fbp"):
        ops = oracle.Operators(g, kind)
        r = krylov.ba_gmres(ops.A, ops.B, b, K, keep_basis=False)
        out["bagmres_" + kind] = {"resid": [float(v) for v in r["resid"]],
                                  "x_final": np.asarray(r["x_final"]).reshape(-1).tolist()}
    return out


def main():
    data = {"generator": "tests/golden/make_oracle_fixture.py",
            "cases": {name: case_outputs(g) for name, g in CASES.items()}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tiny_cases.json")
    with open(path, "w") as f:
        json.dump(data, f, separators=(",", ":"))
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()

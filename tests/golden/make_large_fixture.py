"""Writes the FP64 oracle's solves on the two full-size cone-beam scans, for
the GPU parity tests at those sizes (tests/test_gpu_large.py).  It calls
only ``oracle/`` and the seeded generators of ``ct_inputs.py``.

Cases (one file ``oracle_<case>.npz`` each, beside this script):

* ``c2_ba``, ``c2_ab``, ``c2_cgls``: the 128^3 scan (1 mm voxels, 128 views
  over 360 degrees, 192 x 128 detector of 1.5 mm, sod 500, sdd 1000) with
  noiseless data b = A x_true, x_true the seeded 12-ellipsoid phantom.
  BA-GMRES (Eq. 5) and AB-GMRES (Eq. 4) with B = B_un, 50 iterations each,
  and CGLS(A, B_un) (Eqs. 2-3), 50 iterations, recording the recomputed
  data residual ||b - A x_j|| whose growth shows the divergence of Sec. III
  (Fig. 2).
* ``c3_ba``: the 256^3 scan (0.5 mm voxels, 360 views, 384 x 256 detector
  of 0.75 mm) with Poisson data, counts ~ Poisson(1e5 exp(-A x_true)),
  b = -log(counts/1e5), and BA-GMRES with B = B_FBP (Sec. III), 40
  iterations.
* ``c4_vjp``: the gradient through a converged BA-GMRES solve on the 128^3
  scan (B = B_un): dL/db = B^T z with (A^T B^T) z = g_x, z from 40 GMRES
  iterations on A^T B^T, for a seeded smooth g_x (the "data" here is g_x,
  an image-space vector; the stored sample is of dL/db).

Each case runs the solver twice: once as it is, once with every operator
output multiplied by (1 + 1e-6 N(0,1)) (seeded), the relative error class
of FP32 operators.  The distance between the two runs is the sensitivity
d_k of the k-th iterate to FP32-class operator error, which sets what an
FP32 implementation can be expected to reach.

Stored per case: the geometry, k, the data's norm and a seeded sample of
its entries (so a test that regenerates b can check it has the same data),
the residual history of both runs (and the data residual for CGLS), the
final iterate's norm, the final iterate at a seeded sample of its entries
(voxels; detector readings for the gradient), and d_img = ||x_pert - x|| /
||x|| with the residual sensitivity d_res = max_j |r_pert[j] - r[j]| / r[0].

Run from the repository root (the 256^3 case takes hours on 8 cores):
    python tests/golden/make_large_fixture.py c2_ba c2_ab c2_cgls c3_ba c4_vjp
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ct_inputs as ci  # noqa: E402
import oracle  # noqa: E402
from oracle import krylov  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OP_EPS = 1e-6
PERTURB_SEED = 97
IMAGE_SAMPLES = 20000
IMAGE_SAMPLE_SEED = 5
DATA_SAMPLES = 2000
DATA_SAMPLE_SEED = 6

CASES = {
    "c2_ba": dict(spec="cone_128", solver="ba", b_kind="un", k=50, data="noiseless"),
    "c2_ab": dict(spec="cone_128", solver="ab", b_kind="un", k=50, data="noiseless"),
    "c2_cgls": dict(spec="cone_128", solver="cgls", b_kind="un", k=50, data="noiseless"),
    "c3_ba": dict(spec="cone_256", solver="ba", b_kind="fbp", k=40, data="poisson"),
    "c4_vjp": dict(spec="cone_128", solver="vjp", b_kind="un", k=40, data="smooth_gx"),
}


def case_data(spec, kind):
    """The case's data b (float32, as the GPU receives it) and x_true; for
    the gradient case the image-space vector g_x instead of b."""
    if kind == "smooth_gx":
        return ci.smooth_volume(spec, seed=3).astype(np.float32), None
    x_true = ci.phantom(spec)[0]
    p = oracle.project_A(spec, x_true.astype(np.float64))
    if kind == "poisson":
        b = ci.poisson_log_data(p, i0=1e5, seed=1)
    else:
        b = p.astype(np.float32)
    return b, x_true


def _perturbed(f, rng):
    def g(v):
        y = np.asarray(f(v), dtype=np.float64)
        return y * (1.0 + OP_EPS * rng.standard_normal(y.shape))
    return g


def run_solver(solver, A, B, b64, k):
    if solver == "vjp":   # A, B are A^T, B^T here
        out = krylov.ba_gmres_vjp(A, B, b64, k)
        return dict(resid=np.asarray(out["resid"], dtype=np.float64), x_final=np.asarray(out["gb"]).reshape(-1))
    if solver == "ba":
        out = krylov.ba_gmres(A, B, b64, k, keep_basis=False)
    elif solver == "ab":
        out = krylov.ab_gmres(A, B, b64, k, keep_basis=False)
    else:
        out = krylov.cgls(A, B, b64, k, record_data_resid=True)
    res = dict(resid=np.asarray(out["resid"], dtype=np.float64), x_final=np.asarray(out["x_final"]).reshape(-1))
    if solver == "cgls":
        res["data_resid"] = np.asarray(out["data_resid"], dtype=np.float64)
    return res


def make(name):
    c = CASES[name]
    spec = ci.WORKLOADS[c["spec"]]
    t0 = time.time()
    b, _ = case_data(spec, c["data"])
    b64 = b.astype(np.float64).reshape(-1)
    if c["solver"] == "vjp":
        adj = oracle.AdjointOperators(spec, c["b_kind"])
        op1, op2 = adj.At, adj.Bt
    else:
        ops = oracle.Operators(spec, c["b_kind"])
        op1, op2 = ops.A, ops.B
    ref = run_solver(c["solver"], op1, op2, b64, c["k"])
    t1 = time.time()
    rng = np.random.default_rng(PERTURB_SEED)
    pert = run_solver(c["solver"], _perturbed(op1, rng), _perturbed(op2, rng), b64, c["k"])
    t2 = time.time()
    key = "data_resid" if c["solver"] == "cgls" else "resid"
    x = ref["x_final"]
    # the gradient case's output lives in data space and its input in image space
    vox = ci.sample_indices(x.size, IMAGE_SAMPLES, seed=IMAGE_SAMPLE_SEED)
    rays = ci.sample_indices(b64.size, DATA_SAMPLES, seed=DATA_SAMPLE_SEED)
    meta = dict(case=name, spec=spec.as_dict(), solver=c["solver"], b_kind=c["b_kind"], k=c["k"],
                data=c["data"], op_eps=OP_EPS, perturb_seed=PERTURB_SEED,
                image_sample_seed=IMAGE_SAMPLE_SEED, data_sample_seed=DATA_SAMPLE_SEED,
                oracle_threads=oracle.num_threads(), seconds=[t1 - t0, t2 - t1],
                generator="tests/golden/make_large_fixture.py")
    out = dict(
        meta=np.array(json.dumps(meta)),
        b_norm=np.array(np.linalg.norm(b64)),
        b_sample=b64[rays],
        resid=ref["resid"],
        resid_pert=pert["resid"],
        x_norm=np.array(np.linalg.norm(x)),
        x_sample=x[vox],
        d_img=np.array(np.linalg.norm(pert["x_final"] - x) / np.linalg.norm(x)),
        d_res=np.array(np.max(np.abs(pert[key] - ref[key])) / ref[key][0]),
    )
    if c["solver"] == "cgls":
        out["data_resid"] = ref["data_resid"]
        out["data_resid_pert"] = pert["data_resid"]
    path = os.path.join(HERE, "oracle_%s.npz" % name)
    np.savez_compressed(path, **out)
    print("%s: %.0f s + %.0f s, d_img %.2e, d_res %.2e -> %s" % (name, t1 - t0, t2 - t1, out["d_img"],
                                                                 out["d_res"], path), flush=True)


def main(argv):
    names = argv or list(CASES)
    for n in names:
        if n not in CASES:
            raise SystemExit("unknown case %s (have %s)" % (n, ", ".join(CASES)))
    for n in names:
        make(n)


if __name__ == "__main__":
    main(sys.argv[1:])

"""GPU parity at full size against the FP64 oracle's stored solves
(tests/golden/oracle_<case>.npz, written by make_large_fixture.py, which
calls only the oracle and the seeded generators):

* the 128^3 scan (128 views, 192 x 128 detector, noiseless data):
  BA-GMRES and AB-GMRES with B_un, 50 iterations (Eqs. 4-5), and CGLS(A,
  B_un), 50 iterations (Eqs. 2-3), whose recomputed data residual is
  compared and whose divergence, if the oracle shows one, must show too
  (Sec. III, Fig. 2);
* the 256^3 scan (360 views, 384 x 256 detector, Poisson data from 1e5
  photons): BA-GMRES with B_FBP, 40 iterations, the benchmarked solve;
* the gradient through a converged BA-GMRES solve on the 128^3 scan (B_un):
  40 iterations of GMRES on A^T B^T for a seeded smooth dL/dx, then B^T.

Each test regenerates the data b as the generator did (the oracle's A of
the seeded phantom, then the seeded Poisson draw) and first checks that it
is the stored data (its norm and a seeded sample of entries), then runs the
CUDA solve through the C-ABI in the benchmark's launch configuration and
compares, element by element, the residual history and the final image on
the stored seeded sample of voxels (and its norm).  The bar is the solver
bar of the other parity tests: 1e-4 relative (residuals relative to
resid[0]), or 3 d_k for a case listed in EXCEPTIONS, d_k being the stored
sensitivity of the oracle's own k-th iterate to FP32-class (1e-6) operator
error.
"""
import json
import os

import numpy as np
import pytest
import torch

import ct_inputs as ci
import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SOLVE_TOL = 1e-4

# case -> why its output is held to 3 d_k instead of 1e-4 (measured on a GB300)
EXCEPTIONS = {
    "c4_vjp": "the gradient dL/db after 40 adjoint GMRES iterations at 128^3 (relative residual 0.16): "
              "d_img = 7.9e-4; GPU error 1.25e-4 on the sampled readings, 1.3e-5 on the norm, 2e-7 on "
              "the residual history; A^T and B^T accumulate with FP32 atomics, in an order that varies; "
              "plain FP32 dots 1.24e-4, a second MGS sweep 2.5e-4",
}


def load_case(name):
    path = os.path.join(HERE, "oracle_%s.npz" % name)
    d = np.load(path)
    meta = json.loads(str(d["meta"]))
    return meta, d


@pytest.fixture(scope="module")
def ct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_07408_gb300 import ct as _ct
    return _ct


_DATA = {}


def regenerate_data(meta, d):
    """b as the generator made it (see make_large_fixture.case_data), checked
    against the stored norm and sample."""
    key = (meta["spec"]["name"], meta["data"])
    if key not in _DATA:
        spec = ci.WORKLOADS[meta["spec"]["name"]]
        if meta["data"] == "smooth_gx":
            b = ci.smooth_volume(spec, seed=3).astype(np.float32)
        else:
            x_true = ci.phantom(spec)[0]
            p = oracle.project_A(spec, x_true.astype(np.float64))
            if meta["data"] == "poisson":
                b = ci.poisson_log_data(p, i0=1e5, seed=1)
            else:
                b = p.astype(np.float32)
        _DATA[key] = b
    b = _DATA[key]
    b64 = b.astype(np.float64).reshape(-1)
    rays = ci.sample_indices(b64.size, d["b_sample"].size, seed=meta["data_sample_seed"])
    assert abs(np.linalg.norm(b64) - float(d["b_norm"])) <= 1e-9 * float(d["b_norm"]), \
        "the regenerated data differ from the stored ones (norm)"
    mism = np.count_nonzero(b64[rays] != d["b_sample"])
    assert mism <= 2, "the regenerated data differ from the stored ones at %d of %d samples" % (mism, rays.size)
    return b


def errors(meta, d, x_gpu, resid_gpu, key="resid"):
    ref = d[key]
    k = meta["k"]
    r = np.asarray(resid_gpu[:k + 1], dtype=np.float64)
    err_res = float(np.max(np.abs(r - ref)) / ref[0])
    vox = ci.sample_indices(x_gpu.numel(), d["x_sample"].size, seed=meta["image_sample_seed"])
    xs = x_gpu.reshape(-1)[torch.from_numpy(vox).to(x_gpu.device)].double().cpu().numpy()
    err_img = float(np.linalg.norm(xs - d["x_sample"]) / np.linalg.norm(d["x_sample"]))
    err_norm = abs(float(x_gpu.double().norm()) - float(d["x_norm"])) / float(d["x_norm"])
    return err_img, err_res, err_norm


def compare(parity_log, name, meta, d, x_gpu, resid_gpu, key="resid", rerun=None):
    """Logs and checks one case; ``rerun(**opts)`` -> (x, resid) reruns the
    GPU solve with plain FP32 dots or a second MGS sweep, for the record,
    when an error passes 1e-4."""
    k = meta["k"]
    exc = EXCEPTIONS.get(name)
    d_img, d_res = float(d["d_img"]), float(d["d_res"])
    tol_x = max(SOLVE_TOL, 3 * d_img) if exc else SOLVE_TOL
    tol_r = max(SOLVE_TOL, 3 * d_res) if exc else SOLVE_TOL
    err_img, err_res, err_norm = errors(meta, d, x_gpu, resid_gpu, key)
    variants = {}
    if rerun is not None and max(err_img, err_res, err_norm) > SOLVE_TOL:
        for vname, opts in (("dot_mode=1", dict(dot_mode=1)), ("reorth=1", dict(reorth=1))):
            e = errors(meta, d, *rerun(**opts), key=key)
            variants[vname] = {"err_img": e[0], "err_res": e[1], "err_norm": e[2]}
    parity_log(k=k, d_img=d_img, d_res=d_res, tol_x=tol_x, tol_r=tol_r, err_img=err_img, err_res=err_res,
               err_norm=err_norm, exception=bool(exc), solver=meta["solver"], case=name, b_kind=meta["b_kind"],
               variants=variants)
    assert err_res <= tol_r, ("residual history", err_res, tol_r)
    assert err_img <= tol_x, ("image (sampled voxels)", err_img, tol_x)
    assert err_norm <= tol_x, ("image norm", err_norm, tol_x)
    return err_img, err_res


@pytest.mark.parametrize("name", ["c2_ba", "c2_ab", "c3_ba"])
def test_gmres_matches_stored_oracle_solve(ct, parity_log, name):
    meta, d = load_case(name)
    spec = ci.WORKLOADS[meta["spec"]["name"]]
    b = regenerate_data(meta, d)
    g = ct.Geometry.from_spec(spec)
    bd = torch.from_numpy(b).cuda()
    x = torch.empty(spec.vol_shape, device="cuda")
    opts = ct.make_opts(b_kind=meta["b_kind"])
    solve = ct.ct_bagmres_solve if meta["solver"] == "ba" else ct.ct_abgmres_solve
    res = solve(g, bd, meta["k"], x, opts)
    assert res.iters == meta["k"]
    assert np.all(np.diff(res.resid) <= 1e-6 * res.resid[0])
    compare(parity_log, name, meta, d, x, res.resid)


def test_cgls_unmatched_matches_stored_oracle_and_its_divergence(ct, parity_log):
    name = "c2_cgls"
    meta, d = load_case(name)
    spec = ci.WORKLOADS[meta["spec"]["name"]]
    b = regenerate_data(meta, d)
    g = ct.Geometry.from_spec(spec)
    x = torch.empty(spec.vol_shape, device="cuda")
    res = ct.ct_cgls_solve(g, torch.from_numpy(b).cuda(), meta["k"], x,
                           ct.make_opts(b_kind=meta["b_kind"], record_data_resid=True))
    assert res.iters == meta["k"]
    compare(parity_log, name, meta, d, x, res.resid, key="data_resid")
    # Sec. III (Fig. 2): with the unmatched pair the data residual of CGLS
    # reaches a minimum and then grows; the stored oracle solve of this scan
    # has its minimum at iteration 26 and ends 8.7x above it, and the GPU
    # must show the same
    ref = d["data_resid"]
    r = res.resid[:meta["k"] + 1]
    j_ref, j_gpu = int(np.argmin(ref)), int(np.argmin(r))
    parity_log(k=meta["k"], case=name, oracle_min_at=j_ref, gpu_min_at=j_gpu,
               oracle_final_over_min=float(ref[-1] / ref[j_ref]), gpu_final_over_min=float(r[-1] / r[j_gpu]))
    assert 0 < j_ref < meta["k"] and ref[-1] > 2 * ref[j_ref]
    assert j_gpu == j_ref and r[-1] > 2 * r[j_gpu]


def test_vjp_matches_stored_oracle_gradient(ct, parity_log):
    """The gradient through a converged BA-GMRES solve at 128^3 (Sec. II,
    Eq. 5): dL/db = B^T z, (A^T B^T) z = dL/dx, 40 iterations of GMRES on
    A^T B^T for the seeded smooth dL/dx of the stored oracle case; dL/db on
    its 20 000 stored detector readings, its norm and the residual history."""
    name = "c4_vjp"
    meta, d = load_case(name)
    spec = ci.WORKLOADS[meta["spec"]["name"]]
    gx = regenerate_data(meta, d)
    g = ct.Geometry.from_spec(spec)
    gb = torch.empty(spec.sino_shape, device="cuda")
    gxd = torch.from_numpy(gx.reshape(spec.vol_shape)).cuda()
    res = ct.ct_bagmres_vjp(g, gxd, meta["k"], gb, ct.make_opts(b_kind=meta["b_kind"]))
    assert res.iters == meta["k"]

    def rerun(**o):
        out = torch.empty_like(gb)
        rr = ct.ct_bagmres_vjp(g, gxd, meta["k"], out, ct.make_opts(b_kind=meta["b_kind"], **o))
        return out, rr.resid
    compare(parity_log, name, meta, d, gb, res.resid, rerun=rerun)

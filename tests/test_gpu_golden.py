"""The CUDA path against the oracle's stored outputs on two tiny scans
(tests/golden/oracle_tiny_cases.json, written by the oracle alone): a 2D
parallel-beam scan (8 x 8 pixels, 12 views, 13 bins) and a cone-beam scan
(8^3 voxels, 12 views, 13 x 9 detector), sizes below one tile of every
kernel.

The operators meet the operator bar (relative L2 1e-5, FP32 against FP64).
BA-GMRES is checked on what the method minimises: the residual history
within 1e-4 of ||Bb||, and the oracle's own ||B(b - A x_k)|| of the GPU's
final iterate equal to the GPU's last residual within the same bound.
"""
import json
import os

import numpy as np
import pytest
import torch

import ct_inputs as ci
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_tiny_cases.json")
with open(GOLDEN) as f:
    DATA = json.load(f)
OP_TOL = 1e-5
RESID_TOL = 1e-4


@pytest.fixture(scope="module")
def ct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_07408_gb300 import ct as _ct
    return _ct


def geometry(name):
    return ci.Geometry(name=name, **DATA["cases"][name]["spec"])


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a, shape):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).reshape(shape), dtype=np.float32)).cuda()


@pytest.mark.parametrize("name", sorted(DATA["cases"]))
def test_operators_match_stored_oracle_outputs(ct, name):
    c = DATA["cases"][name]
    spec = geometry(name)
    g = ct.Geometry.from_spec(spec)
    x = ci.random_vector(spec.n, c["x_seed"], positive=True)
    y = ci.random_vector(spec.m, c["y_seed"], positive=True)
    assert rel(ct.project_A(g, dev(x, spec.vol_shape)).cpu().numpy(), c["Ax"]) <= OP_TOL
    assert rel(ct.backproject_B(g, dev(y, spec.sino_shape), "un").cpu().numpy(), c["Bun_y"]) <= OP_TOL
    assert rel(ct.backproject_B(g, dev(y, spec.sino_shape), "fbp").cpu().numpy(), c["Bfbp_y"]) <= OP_TOL


@pytest.mark.parametrize("name", sorted(DATA["cases"]))
@pytest.mark.parametrize("kind", ["un", "fbp"])
def test_bagmres_matches_stored_oracle_history(ct, name, kind):
    c = DATA["cases"][name]
    spec = geometry(name)
    g = ct.Geometry.from_spec(spec)
    b = np.asarray(c["Ax"])
    ref = np.asarray(c["bagmres_" + kind]["resid"])
    x, res = ct.bagmres(g, dev(b, spec.sino_shape), c["k"], b_kind=kind)
    assert res.iters == c["k"]
    got = np.asarray(res.resid[:c["k"] + 1])
    assert np.max(np.abs(got - ref)) <= RESID_TOL * ref[0], (got, ref)
    ops = oracle.Operators(spec, kind)
    xk = x.cpu().double().numpy().reshape(-1)
    true_resid = np.linalg.norm(ops.B(b - ops.A(xk)))
    assert abs(true_resid - got[-1]) <= RESID_TOL * ref[0], (true_resid, got[-1])

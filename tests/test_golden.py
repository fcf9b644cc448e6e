"""The oracle against its stored outputs on two tiny scans
(tests/golden/oracle_tiny_cases.json, written by
tests/golden/make_oracle_fixture.py from the oracle alone).

A regression guard: it fails when the oracle's arithmetic changes.  The
oracle's pins against the mathematics are in tests/test_oracle_*.py.
"""
import json
import os

import numpy as np
import pytest

import ct_inputs as ci
import oracle
from oracle import krylov

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_tiny_cases.json")
with open(GOLDEN) as f:
    DATA = json.load(f)


def geometry(name):
    return ci.Geometry(name=name, **DATA["cases"][name]["spec"])


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name", sorted(DATA["cases"]))
def test_oracle_operators_reproduce_stored_outputs(name):
    c = DATA["cases"][name]
    g = geometry(name)
    x = ci.random_vector(g.n, c["x_seed"], positive=True)
    y = ci.random_vector(g.m, c["y_seed"], positive=True)
    # the C oracle evaluates every output in a fixed order (FP64, no contraction)
    assert rel(oracle.project_A(g, x), c["Ax"]) <= 1e-13
    assert rel(oracle.backproject_B(g, y), c["Bun_y"]) <= 1e-13
    assert rel(oracle.backproject_B(g, y, filtered=True), c["Bfbp_y"]) <= 1e-13


@pytest.mark.parametrize("name", sorted(DATA["cases"]))
@pytest.mark.parametrize("kind", ["un", "fbp"])
def test_oracle_bagmres_reproduces_stored_history(name, kind):
    c = DATA["cases"][name]
    g = geometry(name)
    ops = oracle.Operators(g, kind)
    r = krylov.ba_gmres(ops.A, ops.B, np.asarray(c["Ax"]), c["k"], keep_basis=False)
    ref = c["bagmres_" + kind]
    # numpy's BLAS may order the inner products differently on another host
    assert np.allclose(r["resid"], ref["resid"], rtol=1e-9, atol=0.0)
    assert rel(r["x_final"], ref["x_final"]) <= 1e-8

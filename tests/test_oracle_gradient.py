"""Pin of the oracle's gradient through the converged BA-GMRES solve.

x(b) = (BA)^{-1} B b (Sec. II, Eq. 5).  For L = ||x - x_t||^2 the oracle's
ba_gmres_vjp (GMRES on A^T B^T, then B^T) must equal FP64 central finite
differences of L computed with a dense direct solve.  L is quadratic in b,
so a central difference is exact for any step up to rounding: h = 1e-2
gives a tight check; h = 1e-6 is checked too, with the bound its rounding
allows (the solve's rounding, amplified by cond(BA) ~ 1e4, divided by h).
Checked on a tiny 2D problem with dense matrices, for B_un and B_FBP.
"""
import math

import numpy as np
import pytest

import ct_inputs as ci
import oracle
from oracle import krylov

G = ci.Geometry("tiny2d", ci.PARALLEL_2D, 8, 8, 1, 1.0, 12, 0.0, math.pi, 13, 1, 1.0, 1.0)


@pytest.mark.parametrize("b_kind", ["un", "fbp"])
def test_vjp_equals_central_differences(b_kind):
    A = np.stack([oracle.project_A(G, e).reshape(-1) for e in np.eye(G.n)], axis=1)
    B = np.stack([oracle.backproject_B(G, e, filtered=b_kind == "fbp").reshape(-1) for e in np.eye(G.m)], axis=1)
    x_t = ci.random_vector(G.n, 3, positive=True)
    b = A @ x_t + ci.gaussian_noise(G.m, 0.05, seed=4)

    def loss(bb):
        x = np.linalg.solve(B @ A, B @ bb)
        return float(np.sum((x - x_t) ** 2))

    x = np.linalg.solve(B @ A, B @ b)
    gx = 2.0 * (x - x_t)
    adj = oracle.AdjointOperators(G, b_kind)
    out = krylov.ba_gmres_vjp(adj.At, adj.Bt, gx, G.n)
    idx = ci.sample_indices(G.m, 24, seed=2)
    for h, rtol in ((1e-2, 1e-9), (1e-6, 1e-4)):
        fd = np.array([(loss(b + h * e) - loss(b - h * e)) / (2 * h)
                       for e in (np.eye(G.m)[i] for i in idx)])
        np.testing.assert_allclose(out["gb"][idx], fd, rtol=rtol, atol=rtol * np.abs(fd).max())
    # and the dense closed form B^T (BA)^{-T} gx
    dense = B.T @ np.linalg.solve((B @ A).T, gx)
    np.testing.assert_allclose(out["gb"], dense, rtol=1e-8, atol=1e-10 * np.abs(dense).max())

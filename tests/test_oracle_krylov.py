"""Pins of the oracle's BA-GMRES, AB-GMRES and CGLS (CPU only).

Sec. II: BA-GMRES minimises ||BAx - Bb|| over the Krylov space K_j(BA, Bb)
(zero start, first basis vector Bb); AB-GMRES minimises ||ABy - b|| over
K_j(AB, b) with x = By; the basis is orthonormal and grows by one vector per
iteration; the minimised residual cannot increase.  Sec. I: CGLS needs
B = A^T; with an unmatched pair it can diverge (Sec. III, Fig. 2).  Pins:
  * Arnoldi relation S V_k = V_{k+1} H_k and orthonormality of V;
  * residual history non-increasing and equal to the recomputed residual;
  * iterates equal the least-squares minimiser over an explicitly built
    Krylov basis (dense, tiny), and at k = n the direct solve of BAx = Bb;
  * lucky breakdown on an invariant subspace returns the exact solution, and
    on a subspace where the operator is singular the least-squares residual;
  * BA-GMRES iterates do not depend on the scale of B;
  * matched CGLS equals the Krylov least-squares minimiser; unmatched CGLS
    reaches a minimum data residual and then diverges, while BA-GMRES on the
    same data keeps decreasing.
"""
import math

import numpy as np
import pytest

import ct_inputs as ci
import oracle
from oracle import krylov


def dense_ops(g):
    A = np.stack([oracle.project_A(g, e).reshape(-1) for e in np.eye(g.n)], axis=1)
    B = np.stack([oracle.backproject_B(g, e).reshape(-1) for e in np.eye(g.m)], axis=1)
    return A, B


TINY2D = ci.Geometry("tiny2d", ci.PARALLEL_2D, 8, 8, 1, 1.0, 12, 0.0, math.pi, 13, 1, 1.0, 1.0)
TINYCONE = ci._cone("tinycone", 8, 10.0, 12, 13, 9, 14.0, ang0=0.2)
SMALLCONE = ci._cone("smallcone", 16, 8.0, 20, 24, 16, 12.0, ang0=0.1)


@pytest.fixture(scope="module")
def tiny2d():
    A, B = dense_ops(TINY2D)
    x = ci.random_vector(TINY2D.n, 7, positive=True)
    b = A @ x + ci.gaussian_noise(TINY2D.m, 0.01 * (A @ x).max(), seed=8)
    return A, B, b


def krylov_matrix(S, r0, k):
    K = np.zeros((r0.size, k))
    v = r0.copy()
    for j in range(k):
        K[:, j] = v
        v = S @ v
    return K


def test_arnoldi_relation_and_orthonormal_basis():
    g = SMALLCONE
    ops = oracle.Operators(g, "un")
    vol, _ = ci.phantom(g)
    b = ops.A(vol.astype(np.float64))
    k = 20
    out = krylov.ba_gmres(ops.A, ops.B, b, k)
    V, H = out["V"], out["H"]
    assert out["iters"] == k
    SV = np.stack([ops.B(ops.A(V[:, j])) for j in range(k)], axis=1)
    rel = np.linalg.norm(SV - V @ H) / np.linalg.norm(SV)
    assert rel <= 1e-13, rel
    assert np.linalg.norm(np.eye(k + 1) - V.T @ V) <= 1e-10
    # first basis vector is B b normalised (Sec. II, zero initial vector)
    Bb = ops.B(b)
    np.testing.assert_allclose(V[:, 0], Bb / np.linalg.norm(Bb), rtol=0, atol=1e-15)
    assert np.all(np.diag(H, -1) > 0)


@pytest.mark.parametrize("b_kind", ["un", "fbp"])
def test_residual_history_monotone_and_true(b_kind):
    g = SMALLCONE
    ops = oracle.Operators(g, b_kind)
    vol, _ = ci.phantom(g)
    b = ops.A(vol.astype(np.float64))
    b = b + ci.gaussian_noise(b.size, 0.01 * b.max(), seed=9)
    out = krylov.ba_gmres(ops.A, ops.B, b, 15)
    res = out["resid"]
    assert np.all(np.diff(res) <= 1e-12 * res[0])
    Bb = ops.B(b)
    assert abs(res[0] - np.linalg.norm(Bb)) <= 1e-12 * res[0]
    for j, x in enumerate(out["x"], start=1):
        true = np.linalg.norm(ops.B(b - ops.A(x)))
        assert abs(true - res[j]) <= 1e-11 * res[0], (j, true, res[j])
    assert res[-1] < 0.5 * res[0]


def test_ba_gmres_is_krylov_least_squares(tiny2d):
    A, B, b = tiny2d
    S, r0 = B @ A, B @ b
    out = krylov.ba_gmres(lambda v: A @ v, lambda v: B @ v, b, 8)
    for k in range(1, 9):
        Q, _ = np.linalg.qr(krylov_matrix(S, r0, k))
        z, *_ = np.linalg.lstsq(S @ Q, r0, rcond=None)
        ref = Q @ z
        np.testing.assert_allclose(out["x"][k - 1], ref, rtol=1e-7,
                                   atol=1e-7 * np.abs(ref).max())


def test_ba_gmres_full_dimension_is_direct_solve(tiny2d):
    A, B, b = tiny2d
    n = A.shape[1]
    out = krylov.ba_gmres(lambda v: A @ v, lambda v: B @ v, b, n)
    ref = np.linalg.solve(B @ A, B @ b)
    x = out["x_final"]
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)


def test_ab_gmres_is_krylov_least_squares(tiny2d):
    A, B, b = tiny2d
    S = A @ B
    out = krylov.ab_gmres(lambda v: A @ v, lambda v: B @ v, b, 6)
    for k in range(1, 7):
        Q, _ = np.linalg.qr(krylov_matrix(S, b, k))
        z, *_ = np.linalg.lstsq(S @ Q, b, rcond=None)
        y = Q @ z
        np.testing.assert_allclose(out["x"][k - 1], B @ y, rtol=1e-7,
                                   atol=1e-7 * np.abs(B @ y).max())
        assert abs(out["resid"][k] - np.linalg.norm(A @ (B @ y) - b)) < 1e-9 * out["resid"][0]


def test_lucky_breakdown_gives_exact_solution():
    d = np.arange(1.0, 11.0)
    r0 = np.zeros(10)
    r0[[1, 4, 7]] = [1.0, -2.0, 0.5]
    out = krylov.gmres_core(lambda v: d * v, r0, 10)
    assert out["breakdown"] and out["iters"] == 3
    np.testing.assert_allclose(out["z"][-1], r0 / d, rtol=1e-12, atol=1e-14)
    assert out["resid"][-1] <= 1e-12


def test_breakdown_on_a_singular_operator_keeps_the_least_squares_residual():
    """When the Krylov space becomes invariant and the operator is singular
    on it, the new Hessenberg column vanishes after the rotations: the
    minimum of ||r0 - S z|| over the space is reached at the previous
    iterate and stays above zero.  Brute force (dense least squares over the
    explicit Krylov basis) fixes the history: S = 0 keeps ||r0||; S =
    diag(1, 0) with r0 = (1, 1) gives sqrt 2, then 1 and 1 (S z = (z_1, 0)
    never reaches the second component)."""
    r0 = np.array([0.3, -1.2, 2.0])
    out = krylov.gmres_core(lambda v: 0.0 * v, r0, 3)
    assert out["breakdown"] and out["iters"] == 1
    np.testing.assert_allclose(out["resid"], [np.linalg.norm(r0)] * 2, rtol=1e-15)
    assert np.all(out["z"][-1] == 0.0)
    S = np.diag([1.0, 0.0])
    r0 = np.array([1.0, 1.0])
    out = krylov.gmres_core(lambda v: S @ v, r0, 4)
    assert out["breakdown"] and out["iters"] == 2
    for j in (1, 2):
        K = krylov_matrix(S, r0, j)
        c = np.linalg.lstsq(S @ K, r0, rcond=None)[0]
        assert abs(out["resid"][j] - np.linalg.norm(r0 - S @ K @ c)) <= 1e-12
        np.testing.assert_allclose(S @ out["z"][j - 1], S @ K @ c, atol=1e-12)
        assert np.all(np.isfinite(out["z"][j - 1]))
    np.testing.assert_allclose(out["resid"], [math.sqrt(2.0), 1.0, 1.0], rtol=1e-12)


def test_ba_gmres_iterates_independent_of_B_scale(tiny2d):
    A, B, b = tiny2d
    o1 = krylov.ba_gmres(lambda v: A @ v, lambda v: B @ v, b, 6)
    o2 = krylov.ba_gmres(lambda v: A @ v, lambda v: 3.7 * (B @ v), b, 6)
    for x1, x2 in zip(o1["x"], o2["x"]):
        np.testing.assert_allclose(x1, x2, rtol=1e-9, atol=1e-12)


def test_cgls_matched_is_krylov_least_squares(tiny2d):
    A, _, b = tiny2d
    out = krylov.cgls(lambda v: A @ v, lambda v: A.T @ v, b, 8, record_data_resid=True)
    S, r0 = A.T @ A, A.T @ b
    for k in range(1, 9):
        Q, _ = np.linalg.qr(krylov_matrix(S, r0, k))
        z, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        np.testing.assert_allclose(out["x"][k - 1], Q @ z, rtol=1e-7,
                                   atol=1e-7 * np.abs(Q @ z).max())
    assert np.all(np.diff(out["resid"]) <= 1e-12 * out["resid"][0])
    np.testing.assert_allclose(out["resid"], out["data_resid"], rtol=1e-9)


def test_unmatched_cgls_diverges_while_ba_gmres_converges():
    """Sec. III, Fig. 2: CGLS with (A, B_un) first lowers ||Ax - b||, then
    diverges; BA-GMRES on the same data lowers ||BAx - Bb|| monotonically."""
    g = TINYCONE
    A, B = dense_ops(g)
    x = ci.random_vector(g.n, 1, positive=True)
    b = A @ x
    out = krylov.cgls(lambda v: A @ v, lambda v: B @ v, b, 50, record_data_resid=True)
    data = out["data_resid"]
    jmin = int(np.argmin(data))
    assert 0 < jmin < 40
    assert data[-1] > 10 * data[jmin]
    # the unmatched pair is what breaks it: B = A^T converges on the same data
    ok = krylov.cgls(lambda v: A @ v, lambda v: A.T @ v, b, 50)
    assert np.all(np.diff(ok["resid"]) <= 1e-12 * ok["resid"][0])
    ba = krylov.ba_gmres(lambda v: A @ v, lambda v: B @ v, b, 50)
    assert np.all(np.diff(ba["resid"]) <= 1e-12 * ba["resid"][0])
    assert ba["resid"][-1] < 1e-3 * ba["resid"][0]


def test_restarted_ba_gmres_is_a_sequence_of_krylov_least_squares(tiny2d):
    """GMRES(m), Sec. II: each cycle's correction is the least-squares
    minimiser of ||B r_c - B A dx|| over K_m(BA, B r_c), r_c = b - A x_c,
    built here from an explicit Krylov matrix; the history is the
    concatenation of the cycles' residuals, non-increasing, and its cycle
    ends equal the recomputed ||B (b - A x)||."""
    A, B, b = tiny2d
    m, cycles = 4, 3
    out = krylov.ba_gmres_restarted(lambda v: A @ v, lambda v: B @ v, b, m, cycles)
    S = B @ A
    x = np.zeros(A.shape[1])
    for c in range(cycles):
        rc = B @ (b - A @ x)
        Q, _ = np.linalg.qr(krylov_matrix(S, rc, m))
        z, *_ = np.linalg.lstsq(S @ Q, rc, rcond=None)
        x = x + Q @ z
        assert abs(out["resid"][(c + 1) * m] - np.linalg.norm(B @ (b - A @ x))) <= 1e-10 * out["resid"][0]
    np.testing.assert_allclose(out["x_final"], x, rtol=1e-7, atol=1e-7 * np.abs(x).max())
    assert out["resid"].size == m * cycles + 1
    assert np.all(np.diff(out["resid"]) <= 1e-12 * out["resid"][0])


def test_restarted_single_cycle_is_plain_ba_gmres(tiny2d):
    A, B, b = tiny2d
    plain = krylov.ba_gmres(lambda v: A @ v, lambda v: B @ v, b, 6)
    rest = krylov.ba_gmres_restarted(lambda v: A @ v, lambda v: B @ v, b, 6, 1)
    np.testing.assert_allclose(rest["x_final"], plain["x_final"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(rest["resid"], plain["resid"], rtol=1e-12)

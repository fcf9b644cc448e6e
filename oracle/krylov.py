"""FP64 Krylov solvers of the oracle (test infrastructure only).

BA-GMRES solves B A x = B b (Eq. 5) and AB-GMRES solves A B y = b, x = B y
(Eq. 4), both from a zero initial vector, so the first basis vector is B b
or b (Sec. II).  Each iteration applies the square matrix (BA or AB) to the
newest basis vector, orthonormalises the result against the basis with
modified Gram-Schmidt (Arnoldi), and finds the minimum-residual point of the
grown Krylov subspace, so the residual ||BAx - Bb|| (or ||ABy - b||) never
increases (Sec. II).  The minimum-residual problem is solved with Givens
rotations on the Hessenberg matrix.

CGLS (Eqs. 2-3) is the conjugate-gradient method for min ||Ax - b||; it
assumes B = A^T.  With an unmatched B it is not well defined (Sec. I) and it
is run here only to show what happens.

The solvers take any pair of flat-vector callables, so the tests can also
drive them with explicit dense matrices.
"""
from __future__ import annotations

import math

import numpy as np

BREAKDOWN_RTOL = 1e-14


def _givens(a, b):
    """Rotation (c, s) with [c s; -s c] [a; b] = [r; 0], r = hypot(a, b) >= 0."""
    r = math.hypot(a, b)
    if r == 0.0:
        return 1.0, 0.0, 0.0
    return a / r, b / r, r


def gmres_core(S, r0, k, keep_basis=True):
    """k steps of GMRES on S z = r0 from z0 = 0.

    Returns dict with
      resid: (iters+1,) residual norms ||r0 - S z_j|| (resid[0] = ||r0||),
      z:     list of the iterates z_j, j = 1..iters (z_j in span V_j),
      V:     (len, iters+1) orthonormal basis (if keep_basis),
      H:     (iters+1, iters) Hessenberg matrix of the Arnoldi relation
             S V_iters = V_{iters+1} H,
      iters: iterations done (< k only on a lucky breakdown),
      breakdown: True when the Krylov space became invariant.
    """
    r0 = np.asarray(r0, dtype=np.float64).reshape(-1)
    beta = float(np.linalg.norm(r0))
    n = r0.size
    resid = [beta]
    if beta == 0.0:
        return dict(resid=np.array(resid), z=[], V=np.zeros((n, 1)), H=np.zeros((1, 0)),
                    iters=0, breakdown=True)
    V = np.zeros((n, k + 1))
    V[:, 0] = r0 / beta
    H = np.zeros((k + 1, k))
    R = np.zeros((k + 1, k))       # H after the rotations (upper triangular part)
    cs = np.zeros(k)
    sn = np.zeros(k)
    g = np.zeros(k + 1)
    g[0] = beta
    iters = 0
    breakdown = False
    for j in range(k):
        w = np.asarray(S(V[:, j]), dtype=np.float64).reshape(-1).copy()
        w_norm0 = float(np.linalg.norm(w))
        # modified Gram-Schmidt: project out one basis vector at a time
        for i in range(j + 1):
            H[i, j] = float(np.dot(w, V[:, i]))
            w -= H[i, j] * V[:, i]
        H[j + 1, j] = float(np.linalg.norm(w))
        breakdown = H[j + 1, j] <= BREAKDOWN_RTOL * w_norm0
        if not breakdown:
            V[:, j + 1] = w / H[j + 1, j]
        # rotate the new column by the earlier rotations, then annihilate H[j+1, j]
        col = H[:j + 2, j].copy()
        if breakdown:
            col[j + 1] = 0.0
        for i in range(j):
            t = cs[i] * col[i] + sn[i] * col[i + 1]
            col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1]
            col[i] = t
        cs[j], sn[j], rjj = _givens(col[j], col[j + 1])
        col[j] = rjj
        col[j + 1] = 0.0
        R[:j + 2, j] = col
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        # the least-squares residual is |g[j+1]| while R[j, j] != 0; a column
        # that vanishes after the rotations (only on breakdown: S is singular
        # on the invariant space) cannot reduce g[j], which then stays
        resid.append(abs(g[j + 1]) if rjj != 0.0 else math.hypot(g[j], g[j + 1]))
        iters = j + 1
        if breakdown:
            break
    zs = []
    for j in range(1, iters + 1):
        y = _back_substitute(R[:j, :j], g[:j])
        zs.append(V[:, :j] @ y)
    out = dict(resid=np.array(resid), z=zs, H=H[:iters + 1, :iters], iters=iters,
               breakdown=breakdown, y=_back_substitute(R[:iters, :iters], g[:iters]))
    out["V"] = V[:, :iters + 1] if keep_basis else None
    return out


def _back_substitute(R, g):
    """y = R^{-1} g for upper-triangular R; a zero diagonal entry (the
    vanished column of a singular breakdown) gets y[i] = 0, the minimum-norm
    least-squares choice."""
    k = R.shape[0]
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:] @ y[i + 1:]) / R[i, i] if R[i, i] != 0.0 else 0.0
    return y


def ba_gmres(A, B, b, k, keep_basis=True):
    """BA-GMRES (Eq. 5): minimise ||B A x - B b|| over x in K_j(BA, Bb).

    Returns the gmres_core dict with x (= z) iterates under key "x" and the
    final iterate under "x_final"."""
    r0 = B(np.asarray(b, dtype=np.float64).reshape(-1))
    out = gmres_core(lambda v: B(A(v)), r0, k, keep_basis)
    out["x"] = out["z"]
    out["x_final"] = out["z"][-1] if out["z"] else np.zeros_like(r0)
    return out


def ba_gmres_restarted(A, B, b, m, cycles):
    """Restarted BA-GMRES(m) (Sec. II): cycle c runs m BA-GMRES iterations on
    B A dx = B (b - A x_c) from dx = 0 and sets x_{c+1} = x_c + dx, x_0 = 0.

    Returns dict(x_final, resid) with resid[0] = ||B b|| followed by each
    cycle's residuals ||B (b - A x)|| after its iterations 1..m; a cycle
    that ends early (lucky breakdown) ends the solve."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    x = None
    resid = []
    for c in range(cycles):
        r = b if x is None else b - np.asarray(A(x)).reshape(-1)
        out = ba_gmres(A, B, r, m, keep_basis=False)
        dx = out["x_final"]
        x = dx if x is None else x + dx
        if c == 0:
            resid.append(out["resid"][0])
        resid.extend(out["resid"][1:])
        if out["iters"] < m:
            break
    return dict(x_final=x, resid=np.array(resid))


def ab_gmres(A, B, b, k, keep_basis=True):
    """AB-GMRES (Eq. 4): minimise ||A B y - b|| over y in K_j(AB, b); x = B y."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    out = gmres_core(lambda v: A(B(v)), b, k, keep_basis)
    out["y_iter"] = out["z"]
    out["x"] = [np.asarray(B(y)).reshape(-1) for y in out["z"]]
    out["x_final"] = out["x"][-1] if out["x"] else None
    return out


def cgls(A, B, b, k, record_data_resid=False):
    """CGLS with back-projector B (B = A^T gives the textbook method).

    resid[j] = ||r_j|| where r is updated recursively (r_j = b - A x_j in
    exact arithmetic for any B); data_resid[j] = ||b - A x_j|| recomputed."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    r = b.copy()
    s = np.asarray(B(r)).reshape(-1)
    x = np.zeros_like(s)
    p = s.copy()
    gamma = float(s @ s)
    resid = [float(np.linalg.norm(r))]
    data = [resid[0]]
    xs = []
    for _ in range(k):
        q = np.asarray(A(p)).reshape(-1)
        delta = float(q @ q)
        if delta == 0.0 or gamma == 0.0:
            break
        alpha = gamma / delta
        x = x + alpha * p
        r = r - alpha * q
        s = np.asarray(B(r)).reshape(-1)
        gamma_new = float(s @ s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        resid.append(float(np.linalg.norm(r)))
        if record_data_resid:
            data.append(float(np.linalg.norm(b - np.asarray(A(x)).reshape(-1))))
        xs.append(x.copy())
    return dict(x=xs, x_final=x, resid=np.array(resid),
                data_resid=np.array(data) if record_data_resid else None)


def ba_gmres_vjp(At, Bt, gx, k):
    """Gradient through the converged BA-GMRES solution x = (BA)^{-1} B b:
    dL/db = B^T z with (A^T B^T) z = gx (gx = dL/dx), z from k GMRES steps on
    A^T B^T from zero.  Returns dict(gb, resid, iters)."""
    gx = np.asarray(gx, dtype=np.float64).reshape(-1)
    out = gmres_core(lambda v: At(Bt(v)), gx, k, keep_basis=False)
    z = out["z"][-1] if out["z"] else np.zeros_like(gx)
    return dict(gb=np.asarray(Bt(z)).reshape(-1), resid=out["resid"], iters=out["iters"], z=z)

"""Pins of the oracle's projector A and its transpose A^T (CPU only).

A models line integration (Sec. I Eq. 1); the build reads the paper's
ray-driven projector as Joseph's method (one bilinear sample per voxel-centre
plane of the dominant axis).  Pins:
  * A 1 = chord through the plane stack, N_a vox/|d_a| (unit d), for rays that
    stay inside the grid: checks plane count, step weight, interpolation
    weights summing to one;
  * A f for a linear f equals the exact integral of f over that chord
    (Joseph's midpoint samples integrate linear functions exactly): checks the
    sample positions, hence the geometry and the index order;
  * A of a voxelised ellipsoid phantom converges to the closed-form ellipsoid
    line integrals as the grid is refined;
  * <A x, y> = <x, A^T y> to 1e-12 and, at 8^3, A^T equals the transpose of
    the dense A column by column.
"""
import numpy as np
import pytest

import ct_inputs as ci
import oracle
from oracle import analytic


def plane_samples(g, rays):
    """Fractional grid indices of every Joseph sample of the listed rays,
    from the unit ray direction: returns (a, fb, fz, S, d) with fb, fz of
    shape (R, N_a)."""
    S, d = analytic.ray_geometry(g, rays)
    a = np.where(np.abs(d[:, 0]) >= np.abs(d[:, 1]), 0, 1)
    out_b, out_z = [], []
    for r in range(S.shape[0]):
        ax = a[r]
        bx = 1 - ax
        Na = g.nx if ax == 0 else g.ny
        Nb = g.ny if ax == 0 else g.nx
        c = (np.arange(Na) - (Na - 1) / 2.0) * g.vox
        t = (c - S[r, ax]) / d[r, ax]
        pts = S[r][None, :] + t[:, None] * d[r][None, :]
        out_b.append(pts[:, bx] / g.vox + (Nb - 1) / 2.0)
        out_z.append(pts[:, 2] / g.vox + (g.nz - 1) / 2.0)
    return a, out_b, out_z, S, d


def inside_rays(g, rays):
    a, fb, fz, S, d = plane_samples(g, rays)
    keep = []
    for r in range(len(rays)):
        Nb = g.ny if a[r] == 0 else g.nx
        if (fb[r].min() >= 0 and fb[r].max() <= Nb - 1 and fz[r].min() >= 0
                and fz[r].max() <= g.nz - 1):
            keep.append(r)
    keep = np.array(keep, dtype=np.int64)
    return rays[keep], a[keep], S[keep], d[keep]


GEOMS = [ci.CONE_ANISO, ci.PAR2D_ANISO, ci.CONE_SMALL]


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
def test_A_of_ones_is_chord_length(g):
    rays = ci.sample_indices(g.m, 3000, seed=11)
    rin, a, S, d = inside_rays(g, rays)
    assert rin.size > 100
    y = oracle.project_A_rays(g, np.ones(g.n), rin)
    Na = np.where(a == 0, g.nx, g.ny)
    expect = Na * g.vox / np.abs(d[np.arange(d.shape[0]), a])
    np.testing.assert_allclose(y, expect, rtol=1e-12)


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
def test_A_integrates_linear_functions_exactly(g):
    xs, ys, zs = ci.voxel_centres(g)
    alpha, beta = 0.7, np.array([0.013, -0.021, 0.017])
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    f = alpha + beta[0] * X + beta[1] * Y + beta[2] * Z
    rays = ci.sample_indices(g.m, 3000, seed=12)
    rin, a, S, d = inside_rays(g, rays)
    assert rin.size > 100
    y = oracle.project_A_rays(g, f, rin)
    idx = np.arange(d.shape[0])
    Na = np.where(a == 0, g.nx, g.ny)
    length = Na * g.vox / np.abs(d[idx, a])
    # midpoint of the chord between the outer half-planes = crossing of the
    # central plane (coordinate 0 along the dominant axis)
    t0 = -S[idx, a] / d[idx, a]
    mid = S + t0[:, None] * d
    expect = length * (alpha + mid @ beta)
    np.testing.assert_allclose(y, expect, rtol=1e-11, atol=1e-11 * np.abs(expect).max())


def test_A_converges_to_analytic_line_integrals():
    ells = ci.random_ellipsoids(12, seed=0)
    errs = []
    for nvox in (32, 64, 128):
        g = ci._cone("conv", nvox, 128.0 / nvox, 6, 64, 48, 4.0)
        vol = ci.voxelize(g, ells, dtype=np.float64, supersample=2)
        y = oracle.project_A(g, vol).reshape(-1)
        ya = analytic.ellipsoid_line_integrals(g, ells)
        errs.append(np.linalg.norm(y - ya) / np.linalg.norm(ya))
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.02, errs


def test_A_2d_disc_line_integrals():
    g = ci.PAR2D_64
    disc = [ci.Ellipsoid(np.array([3.0, -2.0, 0.0]), np.array([20.0, 20.0, 1e6]), np.eye(3), 1.0)]
    vol = ci.voxelize(g, disc, dtype=np.float64, supersample=4)
    y = oracle.project_A(g, vol).reshape(-1)
    ya = analytic.ellipsoid_line_integrals(g, disc)
    assert np.linalg.norm(y - ya) / np.linalg.norm(ya) < 0.02


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
def test_At_dot_product(g):
    x = ci.random_vector(g.n, seed=21)
    y = ci.random_vector(g.m, seed=22)
    lhs = float(oracle.project_A(g, x).reshape(-1) @ y)
    rhs = float(x @ oracle.adjoint_At(g, y).reshape(-1))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def tiny_cone():
    return ci._cone("tiny", 8, 10.0, 12, 13, 9, 14.0, ang0=0.2)


def test_At_is_dense_transpose_tiny():
    g = tiny_cone()
    A = np.stack([oracle.project_A(g, e).reshape(-1) for e in np.eye(g.n)], axis=1)
    At = np.stack([oracle.adjoint_At(g, e).reshape(-1) for e in np.eye(g.m)], axis=1)
    np.testing.assert_array_equal(At, A.T)
    assert np.count_nonzero(A) > 0.02 * A.size


def test_A_row_matches_dense_column_order():
    """The (voxel, weight) list of a ray reproduces A applied to unit vectors
    and every weight is positive and at most one step length."""
    g = tiny_cone()
    ray = 12 * 9 // 2 + 6
    idx, w = oracle.a_row(g, ray)
    for j, wj in zip(idx[:5], w[:5]):
        e = np.zeros(g.n)
        e[j] = 1.0
        assert abs(oracle.project_A_rays(g, e, np.array([ray]))[0] - w[idx == j].sum()) < 1e-14
    S, d = analytic.ray_geometry(g, np.array([ray]))
    step = g.vox / np.abs(d[0, :2]).max()
    assert np.all(w > 0) and np.all(w <= step * (1 + 1e-12))

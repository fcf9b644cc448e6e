"""Pins of the oracle's line-intersection projector A_S and its transpose
(CPU only).

Sec. III describes the projector's matrix elements as the intersection
lengths of each ray with the voxels (the line-intersection method); A_S is
that matrix.  Pins, each independent of the oracle's own sort-the-crossings
construction:
  * A_S 1 is the ray's chord through the grid box, found here by bisection
    on a point-in-box test along the ray;
  * A_S x of a random piecewise-constant volume equals brute-force midpoint
    quadrature of x along the ray (a voxel look-up per sample);
  * rays along a grid axis (2D, view angle 0) cross whole pixel columns:
    A_S x = vox times the column sum, exactly;
  * a ray in the central boundary plane of an even grid lies in the
    positive-side slice whatever the FP64 rounding of the grid origin;
  * A_S of a voxelised ellipsoid phantom converges to the closed-form line
    integrals as the grid is refined, and stays close to the Joseph A;
  * <A_S x, y> = <x, A_S^T y> to 1e-12.
"""
import math

import numpy as np
import pytest

import ct_inputs as ci
import oracle
from oracle import analytic

TINY = ci._cone("tinyS", 0, 9.0, 5, 17, 13, 11.0, ang0=0.37, nxyz=(6, 5, 4))
TINY2D = ci.Geometry("tinyS2d", ci.PARALLEL_2D, 7, 6, 1, 1.3, 5, 0.21, math.pi, 11, 1, 1.1, 1.0)
GEOMS = [TINY, TINY2D, ci.CONE_ANISO, ci.PAR2D_ANISO]
SCAN = 20001


def box(g):
    half = 0.5 * np.array([g.nx, g.ny, g.nz]) * g.vox
    return -half, half


def inside(g, pts):
    lo, hi = box(g)
    return np.all((pts > lo) & (pts < hi), axis=-1)


def scan_step(g):
    return 2.02 * float(np.linalg.norm(box(g)[1])) / (SCAN - 1)


def chord_interval(g, S, d):
    """(t_in, t_out) of the ray S + t d (unit d) inside the box: a scan for an
    inside point over the stretch of the ray inside the box's bounding
    sphere, then bisection of the inside test on both sides (the box is
    convex, so the inside set is one interval).  Chords shorter than the scan
    step can be missed (None)."""
    R = float(np.linalg.norm(box(g)[1])) * 1.01
    tc = -float(S @ d)
    ts = np.linspace(tc - R, tc + R, SCAN)
    ins = inside(g, S[None, :] + ts[:, None] * d[None, :])
    if not ins.any():
        return None
    k0, k1 = np.nonzero(ins)[0][[0, -1]]

    def bisect(a, b):   # a inside, b outside
        for _ in range(80):
            m = 0.5 * (a + b)
            if inside(g, S + m * d):
                a = m
            else:
                b = m
        return 0.5 * (a + b)

    t_in = bisect(ts[k0], ts[k0 - 1]) if k0 > 0 else ts[0]
    t_out = bisect(ts[k1], ts[k1 + 1]) if k1 + 1 < ts.size else ts[-1]
    return t_in, t_out


def sample_rays(g, count, seed):
    return ci.sample_indices(g.m, min(count, g.m), seed=seed)


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
def test_AS_of_ones_is_box_chord(g):
    rays = sample_rays(g, 120, 31)
    y = oracle.project_S_rays(g, np.ones(g.n), rays)
    S, d = analytic.ray_geometry(g, rays)    # unit directions
    for r in range(rays.size):
        iv = chord_interval(g, S[r], d[r])
        if iv is None:   # no scan point inside: the chord, if any, is shorter than the step
            assert y[r] < 2 * scan_step(g), (rays[r], y[r])
            continue
        ref = iv[1] - iv[0]
        assert abs(y[r] - ref) <= 1e-9 * max(ref, g.vox), (rays[r], y[r], ref)
    assert np.count_nonzero(y) > rays.size // 3


@pytest.mark.parametrize("g", [TINY, TINY2D], ids=lambda g: g.name)
def test_AS_equals_quadrature_of_piecewise_constant_volume(g):
    x = ci.random_vector(g.n, 33, positive=True).reshape(g.vol_shape)   # x[z][y][x]
    rays = sample_rays(g, 60, 34)
    y = oracle.project_S_rays(g, x.reshape(-1), rays)
    S, d = analytic.ray_geometry(g, rays)
    lo, _ = box(g)
    K = 200000
    for r in range(rays.size):
        iv = chord_interval(g, S[r], d[r])
        if iv is None:
            assert y[r] < 2 * scan_step(g) * x.max()
            continue
        t = iv[0] + (np.arange(K) + 0.5) * (iv[1] - iv[0]) / K
        p = S[r][None, :] + t[:, None] * d[r][None, :]
        i = np.clip(np.floor((p - lo) / g.vox).astype(np.int64), 0, [g.nx - 1, g.ny - 1, g.nz - 1])
        quad = x[i[:, 2], i[:, 1], i[:, 0]].sum() * (iv[1] - iv[0]) / K
        assert abs(y[r] - quad) <= 2e-4 * max(quad, 1e-12), (rays[r], y[r], quad)


def test_AS_axis_aligned_rays_sum_columns():
    g = ci.Geometry("axis2d", ci.PARALLEL_2D, 9, 7, 1, 2.0, 1, 0.0, math.pi, 8, 1, 2.2, 1.0)
    x = ci.random_vector(g.n, 35).reshape(g.ny, g.nx)
    y = oracle.project_S(g, x.reshape(-1)).reshape(-1)
    # view angle 0: ray iu is the line x = u along +y
    for iu in range(g.nu):
        u = (iu - (g.nu - 1) / 2.0) * g.du
        col = math.floor((u + 0.5 * g.nx * g.vox) / g.vox)
        ref = g.vox * x[:, col].sum() if 0 <= col < g.nx else 0.0
        assert abs(y[iu] - ref) <= 1e-12 * max(1.0, abs(ref)), (iu, y[iu], ref)


def test_AS_ray_in_the_central_plane_belongs_to_the_positive_side():
    """Rays of the central detector row of a cone-beam scan lie in the plane
    z = 0, which on a grid of even nz is the boundary between slices
    nz/2 - 1 and nz/2; the reading for such a measure-zero case puts them in
    slice nz/2 (the positive side).  With a voxel edge for which
    (nz/2 vox)/vox rounds below nz/2 in FP64, every voxel of those rows must
    still be in slice nz/2, with the whole chord length."""
    vox = 2.6169519915633814
    assert math.floor((0.5 * 28 * vox) / vox) == 13   # the rounding the reading must not depend on
    g = ci._cone("central_plane", 0, vox, 4, 20, 9, 6.0, nxyz=(11, 9, 28), ang0=0.3)
    ones = oracle.project_S(g, np.ones(g.n)).reshape(g.sino_shape)
    for s in range(g.n_views):
        for iu in range(g.nu):
            ray = (s * g.nv + (g.nv - 1) // 2) * g.nu + iu
            cols, lens = oracle.s_row(g, ray)
            assert np.all(cols // (g.nx * g.ny) == g.nz // 2)
            assert abs(lens.sum() - ones[s, (g.nv - 1) // 2, iu]) <= 1e-9


def test_AS_converges_to_analytic_line_integrals_and_near_joseph():
    ells = ci.random_ellipsoids(12, seed=0)
    errs = []
    for nvox in (32, 64, 128):
        g = ci._cone("convS", nvox, 128.0 / nvox, 6, 64, 48, 4.0)
        vol = ci.voxelize(g, ells, dtype=np.float64, supersample=2)
        ys = oracle.project_S(g, vol).reshape(-1)
        ya = analytic.ellipsoid_line_integrals(g, ells)
        errs.append(np.linalg.norm(ys - ya) / np.linalg.norm(ya))
        if nvox == 128:
            yj = oracle.project_A(g, vol).reshape(-1)
            assert np.linalg.norm(ys - yj) / np.linalg.norm(yj) < 0.02
    # piecewise-constant voxels converge more slowly than Joseph's interpolation
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.03, errs


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
def test_ASt_dot_product(g):
    x = ci.random_vector(g.n, seed=36)
    y = ci.random_vector(g.m, seed=37)
    lhs = float(oracle.project_S(g, x).reshape(-1) @ y)
    rhs = float(x @ oracle.adjoint_St(g, y).reshape(-1))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)

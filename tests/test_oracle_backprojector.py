"""Pins of the oracle's back-projectors B_un, B_FBP = B_un F and their
transposes (CPU only).

B_un is voxel-driven back-projection with linear interpolation on the
detector (Sec. III).  Pins:
  * B_un g for a sinogram g linear in (u, v) on every view equals
    sum_views w * g(u(r), v(r)) with the voxel's detector position found by an
    independent ray/plane intersection (bilinear interpolation is exact on
    linear data): checks projection geometry, weights and index order;
  * B_un ~ A^T (Sec. III): <B_un A x, x> / <A x, A x> close to one;
  * the ramp filter's Ram-Lak kernel has frequency response |w|/(2 pi tau^2):
    a sinusoidal row comes out scaled by that factor;
  * B_FBP applied to the closed-form projections of a disc / ball gives the
    density inside (FBP calibration of c_F);
  * <B y, x> = <y, B^T x> and <F y, z> = <y, F^T z> to 1e-12.
"""
import math

import numpy as np
import pytest

import ct_inputs as ci
import oracle
from oracle import analytic


def detector_positions(g, voxels):
    """(fu, fv, weight) of each voxel in each view by intersecting the
    source->voxel line with the detector plane.  Shapes (V, n_views)."""
    iz = voxels // (g.nx * g.ny)
    iy = (voxels // g.nx) % g.ny
    ix = voxels % g.nx
    xs, ys, zs = ci.voxel_centres(g)
    r = np.stack([xs[ix], ys[iy], zs[iz]], axis=1)            # (V, 3)
    th = g.ang0 + np.arange(g.n_views) * g.span / g.n_views
    fu = np.zeros((r.shape[0], g.n_views))
    fv = np.zeros_like(fu)
    w = np.zeros_like(fu)
    for s, t in enumerate(th):
        c, sn = math.cos(t), math.sin(t)
        nrm = np.array([c, sn, 0.0])
        eu = np.array([-sn, c, 0.0]) if g.kind == 1 else np.array([c, sn, 0.0])
        ev = np.array([0.0, 0.0, 1.0])
        if g.kind == 1:
            S = g.sod * nrm
            D = -(g.sdd - g.sod) * nrm
            tt = ((D - S) @ nrm) / ((r - S[None, :]) @ nrm)    # ray parameter at the detector
            P = S[None, :] + tt[:, None] * (r - S[None, :])
            u = (P - D[None, :]) @ eu
            v = (P - D[None, :]) @ ev
            w[:, s] = g.vox ** 3 * tt ** 2 / (g.du * g.dv)
        else:
            u = r @ eu
            v = np.zeros(r.shape[0])
            w[:, s] = g.vox ** 2 / g.du
        fu[:, s] = u / g.du + (g.nu - 1) / 2.0
        fv[:, s] = v / g.dv + (g.nv - 1) / 2.0
    return fu, fv, w


GEOMS = [ci.CONE_ANISO, ci.PAR2D_ANISO, ci.CONE_SMALL]


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
def test_B_exact_on_linear_sinograms(g):
    rng = np.random.default_rng(31)
    al = rng.uniform(0.5, 1.5, g.n_views)
    be = rng.uniform(-0.02, 0.02, g.n_views)
    ga = rng.uniform(-0.02, 0.02, g.n_views)
    us = (np.arange(g.nu) - (g.nu - 1) / 2.0)
    vs = (np.arange(g.nv) - (g.nv - 1) / 2.0)
    sino = (al[:, None, None] + be[:, None, None] * us[None, None, :]
            + ga[:, None, None] * vs[None, :, None])
    vox = ci.sample_indices(g.n, 2000, seed=32)
    fu, fv, w = detector_positions(g, vox)
    inside = ((fu >= 0) & (fu <= g.nu - 1) & (fv >= 0) & (fv <= g.nv - 1)).all(axis=1)
    assert inside.sum() > 50
    vox = vox[inside]
    fu, fv, w = fu[inside], fv[inside], w[inside]
    lin = (al[None, :] + be[None, :] * (fu - (g.nu - 1) / 2.0)
           + ga[None, :] * (fv - (g.nv - 1) / 2.0))
    expect = (w * lin).sum(axis=1)
    got = oracle.backproject_B_voxels(g, sino, vox)
    np.testing.assert_allclose(got, expect, rtol=1e-11)


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
def test_B_un_is_close_to_At_in_scale(g):
    x = ci.smooth_volume(g)
    y = oracle.project_A(g, x).reshape(-1)
    ratio = float(oracle.backproject_B(g, y).reshape(-1) @ x.reshape(-1)) / float(y @ y)
    assert 0.9 < ratio < 1.1, ratio
    # but B_un is not A^T
    At_y = oracle.adjoint_At(g, y).reshape(-1)
    B_y = oracle.backproject_B(g, y).reshape(-1)
    assert np.linalg.norm(B_y - At_y) > 1e-3 * np.linalg.norm(At_y)


@pytest.mark.parametrize("g", GEOMS, ids=lambda g: g.name)
@pytest.mark.parametrize("filtered", [False, True])
def test_Bt_dot_product(g, filtered):
    x = ci.random_vector(g.n, seed=41)
    y = ci.random_vector(g.m, seed=42)
    lhs = float(oracle.backproject_B(g, y, filtered=filtered).reshape(-1) @ x)
    rhs = float(y @ oracle.adjoint_Bt(g, x, filtered=filtered).reshape(-1))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300)


def test_Bt_is_dense_transpose_tiny():
    g = ci._cone("tiny", 8, 10.0, 12, 13, 9, 14.0, ang0=0.2)
    B = np.stack([oracle.backproject_B(g, e).reshape(-1) for e in np.eye(g.m)], axis=1)
    Bt = np.stack([oracle.adjoint_Bt(g, e).reshape(-1) for e in np.eye(g.n)], axis=1)
    np.testing.assert_array_equal(Bt, B.T)


def test_ramlak_frequency_response():
    tau = 0.7
    g = ci.Geometry("ramp", ci.PARALLEL_2D, 4, 4, 1, 1.0, 1, 0.0, math.pi, 2001, 1, tau, 1.0)
    iu = np.arange(g.nu)
    for freq in (0.05, 0.1, 0.31):
        w = 2 * math.pi * freq
        row = np.cos(w * iu)
        out = oracle.ramp_F(g, row).reshape(-1)
        expect = oracle.ramp_scale(g) * (w / (2 * math.pi * tau * tau)) * row
        mid = slice(700, 1300)
        assert np.max(np.abs(out[mid] - expect[mid])) < 3e-3 * np.max(np.abs(expect))
    # constant rows have (almost) zero ramp response in the interior
    out = oracle.ramp_F(g, np.ones(g.nu)).reshape(-1)
    assert np.max(np.abs(out[700:1300])) < 2e-3 * oracle.ramp_scale(g) / (4 * tau * tau)


def test_ramp_scale_closed_form():
    g = ci.CONE_SMALL
    tau = g.du * g.sod / g.sdd
    cf = (math.pi / g.n_views) * (g.sod / g.sdd) ** 2 * g.du * g.dv / g.vox ** 3
    assert abs(oracle.ramp_scale(g) - cf * tau) < 1e-14 * cf * tau


@pytest.mark.parametrize("g", [ci.PAR2D_ANISO, ci.CONE_SMALL], ids=lambda g: g.name)
def test_Ft_dot_product(g):
    y = ci.random_vector(g.m, seed=51)
    z = ci.random_vector(g.m, seed=52)
    lhs = float(oracle.ramp_F(g, y).reshape(-1) @ z)
    rhs = float(y @ oracle.ramp_Ft(g, z).reshape(-1))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_fbp_reconstructs_disc_density_2d():
    g = ci.scaled(ci.PAR2D_64, n_views=180)
    disc = [ci.Ellipsoid(np.zeros(3), np.array([24.0, 24.0, 1e6]), np.eye(3), 1.0)]
    b = analytic.ellipsoid_line_integrals(g, disc)
    f = oracle.backproject_B(g, b, filtered=True).reshape(g.ny, g.nx)
    xs, ys, _ = ci.voxel_centres(g)
    X, Y = np.meshgrid(xs, ys)
    inner = X ** 2 + Y ** 2 < 15.0 ** 2
    outer = X ** 2 + Y ** 2 > 28.0 ** 2
    assert abs(f[inner].mean() - 1.0) < 0.03
    assert abs(f[outer].mean()) < 0.03


def test_fbp_reconstructs_ball_density_cone():
    g = ci.CONE_SMALL
    ball = [ci.Ellipsoid(np.zeros(3), np.array([30.0, 30.0, 30.0]), np.eye(3), 1.0)]
    b = analytic.ellipsoid_line_integrals(g, ball)
    f = oracle.backproject_B(g, b, filtered=True).reshape(g.vol_shape)
    xs, ys, zs = ci.voxel_centres(g)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    inner = (X ** 2 + Y ** 2 + Z ** 2) < 15.0 ** 2
    assert abs(f[inner].mean() - 1.0) < 0.05


def ray_obliquity(g, s, iu, iv):
    """Cosine of the angle between the ray from the source to pixel (iu, iv)
    of view s and the central ray, from the scan's vectors: source
    S = sod (c, s, 0), detector centre D = -(sdd - sod) (c, s, 0), pixel
    P = D + u e_u + v e_v with e_u = (-s, c, 0), e_v = (0, 0, 1)."""
    th = g.ang0 + s * g.span / g.n_views
    c, sn = math.cos(th), math.sin(th)
    S = g.sod * np.array([c, sn, 0.0])
    D = -(g.sdd - g.sod) * np.array([c, sn, 0.0])
    u = (iu - (g.nu - 1) / 2.0) * g.du
    v = (iv - (g.nv - 1) / 2.0) * g.dv
    d = D + u * np.array([-sn, c, 0.0]) + v * np.array([0.0, 0.0, 1.0]) - S
    central = D - S
    return float(d @ central) / (np.linalg.norm(d) * np.linalg.norm(central))


@pytest.mark.parametrize("g", [ci.CONE_SMALL, ci.CONE_ANISO], ids=lambda g: g.name)
def test_ramp_cosine_weight_from_ray_geometry(g):
    """F = c_F tau H diag(w) with w the cosine of each ray's angle to the
    central ray (FDK weighting, the reading of Sec. III's ramp filter); F^T
    applies w after the convolution.  A unit impulse at pixel (k, iv) is
    filtered into c_F tau h[i - k] w(k, iv) along its row: every output
    divided by w(k, iv) is the same kernel whatever the pixel, the corners
    included (w ~ 0.985 there), and it equals the ramp kernel's centre
    value c_F tau / (4 tau^2) at i = k.  For F^T each output i carries
    w(i, iv) instead.  w is computed here from the source and pixel
    positions, not from the oracle's closed form."""
    tau = g.du * g.sod / g.sdd
    centre = oracle.ramp_scale(g) / (4.0 * tau * tau)
    s = 3
    rows = sorted({0, g.nv // 2, g.nv - 1})
    cols = sorted({0, 1, g.nu // 2, g.nu - 2, g.nu - 1})
    kernels = {}
    w_min = 1.0
    for iv in rows:
        for k in cols:
            e = np.zeros(g.sino_shape)
            e[s, iv, k] = 1.0
            f = oracle.ramp_F(g, e)[s, iv]
            ft = oracle.ramp_Ft(g, e)[s, iv]
            others = np.delete(oracle.ramp_F(g, e).reshape(g.n_views * g.nv, g.nu), s * g.nv + iv, axis=0)
            assert not np.any(others), "F mixes detector rows"
            wk = ray_obliquity(g, s, k, iv)
            wi = np.array([ray_obliquity(g, s, i, iv) for i in range(g.nu)])
            w_min = min(w_min, wk)
            assert abs(f[k] - centre * wk) <= 1e-13 * centre
            # the kernel seen from pixel k: h[d] for d = i - k
            for i in range(g.nu):
                d = i - k
                hd = f[i] / wk
                assert abs(ft[i] - hd * wi[i]) <= 1e-13 * centre, ("F^T weight", iv, k, i)
                if d in kernels:
                    assert abs(hd - kernels[d]) <= 1e-13 * centre, ("F weight", iv, k, i)
                else:
                    kernels[d] = hd
    # the corners are oblique enough that a missing or misplaced weight shows
    assert w_min < 0.99

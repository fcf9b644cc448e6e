"""GPU parity of the operators A, B_un, B_FBP, F, A^T, B^T against the FP64
oracle, through the C-ABI.

Tolerance: relative L2 error <= 1e-5 per operator application (FP32
arithmetic against FP64); the bound is stated in each assertion.  Small
cases are compared element by element over the whole output; the 256^3 and
512^3 scans on sampled rays / voxels that the oracle evaluates one by one.
"""
import math

import numpy as np
import pytest
import torch

import ct_inputs as ci
import oracle

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5

# cone_z40: 40 slices, so the last 16-slice run of the 3D back-projector
# passes nz by 8 (the row margin covers it); cone_aniso: 36 rows of columns
# and 28 slices, ragged against its 32 x 8 x 16 tiles
SMALL = [ci.CONE_SMALL, ci.CONE_ANISO, ci.CONE_THIN, ci.PAR2D_ANISO, ci.PAR2D_64, ci.CONE_GRAD32,
         ci.CONE_512_CUT64, ci.CONE_Z40]


@pytest.fixture(scope="module")
def ct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_07408_gb300 import ct as _ct
    return _ct


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().double().numpy()


def volume_input(spec, kind):
    if kind == "phantom":
        return ci.phantom(spec)[0]
    return ci.random_vector(spec.n, seed=61, positive=True).astype(np.float32).reshape(spec.vol_shape)


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: s.name)
@pytest.mark.parametrize("kind", ["phantom", "random"])
def test_project_A_matches_oracle(ct, spec, kind):
    g = ct.Geometry.from_spec(spec)
    x = volume_input(spec, kind)
    y = host(ct.project_A(g, dev(x)))
    ref = oracle.project_A(spec, x.astype(np.float64))
    assert rel(y, ref) <= OP_TOL, rel(y, ref)
    assert np.max(np.abs(y - ref)) <= 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: s.name)
@pytest.mark.parametrize("b_kind", ["un", "fbp"])
def test_backproject_B_matches_oracle(ct, spec, b_kind):
    g = ct.Geometry.from_spec(spec)
    y = oracle.project_A(spec, ci.phantom(spec)[0].astype(np.float64)).astype(np.float32)
    y = y + ci.gaussian_noise(y.shape, 0.01 * y.max(), seed=62, dtype=np.float32)
    x = host(ct.backproject_B(g, dev(y), b_kind))
    ref = oracle.backproject_B(spec, y.astype(np.float64), filtered=b_kind == "fbp")
    assert rel(x, ref) <= OP_TOL, rel(x, ref)


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: s.name)
@pytest.mark.parametrize("transpose", [False, True])
def test_ramp_F_matches_oracle(ct, spec, transpose):
    g = ct.Geometry.from_spec(spec)
    y = ci.random_vector(spec.m, seed=63).astype(np.float32).reshape(spec.sino_shape)
    out = host(ct.ramp_F(g, dev(y), transpose))
    ref = (oracle.ramp_Ft if transpose else oracle.ramp_F)(spec, y.astype(np.float64))
    assert rel(out, ref) <= OP_TOL, rel(out, ref)


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: s.name)
def test_adjoint_At_matches_oracle(ct, spec):
    g = ct.Geometry.from_spec(spec)
    y = ci.random_vector(spec.m, seed=64).astype(np.float32).reshape(spec.sino_shape)
    x = host(ct.adjoint_At(g, dev(y)))
    ref = oracle.adjoint_At(spec, y.astype(np.float64))
    assert rel(x, ref) <= OP_TOL, rel(x, ref)


@pytest.mark.parametrize("spec", SMALL, ids=lambda s: s.name)
@pytest.mark.parametrize("b_kind", ["un", "fbp"])
def test_adjoint_Bt_matches_oracle(ct, spec, b_kind):
    g = ct.Geometry.from_spec(spec)
    x = ci.random_vector(spec.n, seed=65).astype(np.float32).reshape(spec.vol_shape)
    y = host(ct.adjoint_Bt(g, dev(x), b_kind))
    ref = oracle.adjoint_Bt(spec, x.astype(np.float64), filtered=b_kind == "fbp")
    assert rel(y, ref) <= OP_TOL, rel(y, ref)


@pytest.mark.parametrize("spec", [ci.CONE_SMALL, ci.PAR2D_ANISO], ids=lambda s: s.name)
def test_gpu_adjoint_dot_products(ct, spec):
    """<A x, y> = <x, A^T y> and <B y, x> = <y, B^T x> for the GPU kernels
    themselves (FP32: ~1e-6)."""
    g = ct.Geometry.from_spec(spec)
    x = dev(ci.random_vector(spec.n, seed=66).reshape(spec.vol_shape))
    y = dev(ci.random_vector(spec.m, seed=67).reshape(spec.sino_shape))
    # the bound is relative to the Cauchy-Schwarz scale |Ax| |y|: the inner
    # products of random vectors cancel, so FP32 rounding of the terms is
    # measured against their size, not against the (smaller) sum
    ax = ct.project_A(g, x).double()
    ax_y = float((ax * y.double()).sum())
    x_aty = float((x.double() * ct.adjoint_At(g, y).double()).sum())
    assert abs(ax_y - x_aty) <= 1e-5 * float(ax.norm() * y.double().norm())
    for kind in ("un", "fbp"):
        by = ct.backproject_B(g, y, kind).double()
        by_x = float((by * x.double()).sum())
        y_btx = float((y.double() * ct.adjoint_Bt(g, x, kind).double()).sum())
        assert abs(by_x - y_btx) <= 1e-5 * float(by.norm() * x.double().norm()), kind


def test_zero_inputs_give_exact_zeros(ct):
    spec = ci.CONE_ANISO
    g = ct.Geometry.from_spec(spec)
    assert torch.count_nonzero(ct.project_A(g, torch.zeros(spec.vol_shape, device="cuda"))) == 0
    assert torch.count_nonzero(ct.backproject_B(g, torch.zeros(spec.sino_shape, device="cuda"), "fbp")) == 0


def test_single_voxel_and_single_ray(ct):
    """A delta volume projects to the oracle's column of A; a delta sinogram
    back-projects to the oracle's column of B (sparse structure, exact zeros
    outside the footprint)."""
    spec = ci.CONE_ANISO
    g = ct.Geometry.from_spec(spec)
    j = (spec.nz // 2 * spec.ny + 7) * spec.nx + 31
    e = np.zeros(spec.n, dtype=np.float32)
    e[j] = 1.0
    col = host(ct.project_A(g, dev(e.reshape(spec.vol_shape)))).reshape(-1)
    ref = oracle.project_A(spec, e.astype(np.float64)).reshape(-1)
    assert np.array_equal(col != 0, ref != 0)
    assert rel(col, ref) <= OP_TOL
    r = (spec.n_views // 3 * spec.nv + spec.nv // 2) * spec.nu + 17
    d = np.zeros(spec.m, dtype=np.float32)
    d[r] = 1.0
    colb = host(ct.backproject_B(g, dev(d.reshape(spec.sino_shape)))).reshape(-1)
    refb = oracle.backproject_B(spec, d.astype(np.float64)).reshape(-1)
    assert np.array_equal(colb != 0, refb != 0)
    assert rel(colb, refb) <= OP_TOL


@pytest.mark.parametrize("spec", [ci.CONE_128, ci.CONE_256], ids=lambda s: s.name)
def test_full_size_operators_on_sampled_outputs(ct, spec):
    """The operators at the full 128^3 / 256^3 scans, checked on seeded
    samples of rays and voxels that the oracle evaluates one by one."""
    g = ct.Geometry.from_spec(spec)
    x = ci.phantom(spec)[0]
    y = ct.project_A(g, dev(x))
    rays = ci.sample_indices(spec.m, 3000, seed=68)
    ya = host(y).reshape(-1)[rays]
    ref = oracle.project_A_rays(spec, x.astype(np.float64), rays)
    assert rel(ya, ref) <= OP_TOL, rel(ya, ref)
    yn = host(y).astype(np.float32)
    vox = ci.sample_indices(spec.n, 3000, seed=69)
    xb = host(ct.backproject_B(g, dev(yn))).reshape(-1)[vox]
    refb = oracle.backproject_B_voxels(spec, yn.astype(np.float64), vox)
    assert rel(xb, refb) <= OP_TOL, rel(xb, refb)
    rows = ci.sample_indices(spec.n_views * spec.nv, 200, seed=70)
    f = host(ct.ramp_F(g, dev(yn))).reshape(-1, spec.nu)[rows]
    reff = oracle.ramp_F_rows(spec, yn.astype(np.float64), rows)
    assert rel(f, reff) <= OP_TOL, rel(f, reff)


def test_max_size_512_on_sampled_outputs(ct):
    """The largest scan (512^3 voxels, 720 views, 768x512 detector)."""
    spec = ci.CONE_512
    g = ct.Geometry.from_spec(spec)
    x = ci.random_vector(spec.n, seed=71, positive=True).astype(np.float32)
    xd = dev(x.reshape(spec.vol_shape))
    y = ct.project_A(g, xd)
    del xd
    rays = ci.sample_indices(spec.m, 1000, seed=72)
    ya = host(y).reshape(-1)[rays]
    ref = oracle.project_A_rays(spec, x.astype(np.float64), rays)
    assert rel(ya, ref) <= OP_TOL, rel(ya, ref)
    vox = ci.sample_indices(spec.n, 1000, seed=73)
    xb = ct.backproject_B(g, y)
    xb_s = host(xb).reshape(-1)[vox]
    refb = oracle.backproject_B_voxels(spec, host(y).reshape(-1), vox)
    assert rel(xb_s, refb) <= OP_TOL, rel(xb_s, refb)


def test_operator_errors_are_reported(ct):
    spec = ci.CONE_SMALL
    g = ct.Geometry.from_spec(spec)
    with pytest.raises(ValueError):
        ct.ct_project_A(g, torch.zeros(5, device="cuda"), torch.zeros(spec.m, device="cuda"))
    with pytest.raises(TypeError):
        ct.ct_project_A(g, torch.zeros(spec.n, device="cuda", dtype=torch.float64),
                        torch.zeros(spec.m, device="cuda"))
    with pytest.raises(ct.CTError):
        ct.ct_backproject_B(g, torch.zeros(spec.m, device="cuda"), torch.zeros(spec.n, device="cuda"), 9)
    y = torch.zeros(spec.m, device="cuda")
    with pytest.raises(ct.CTError):
        ct.ct_ramp_F(g, y, y)


# --- line-intersection projector (CT_PROJ_SIDDON) -------------------------------
SIDDON_CASES = [ci.CONE_SMALL, ci.CONE_ANISO, ci.CONE_THIN, ci.PAR2D_ANISO, ci.PAR2D_64]


@pytest.mark.parametrize("spec", SIDDON_CASES, ids=lambda s: s.name)
@pytest.mark.parametrize("kind", ["phantom", "random"])
def test_siddon_A_matches_oracle(ct, spec, kind):
    g = ct.Geometry.from_spec(spec, projector="siddon")
    x = volume_input(spec, kind)
    y = host(ct.project_A(g, dev(x)))
    ref = oracle.project_S(spec, x.astype(np.float64))
    assert rel(y, ref) <= OP_TOL, rel(y, ref)


# Line-intersection lengths are ill-conditioned where a ray runs nearly
# parallel to a grid plane: a position error e moves the crossing of that
# plane by e/|h_a| along the ray (h the unit direction).  FP32 ray
# coordinates carry e ~ 1e-6 voxel, so single voxel lengths differ from the
# FP64 oracle's by up to ~1e-4 voxel (a float32 emulation of the walk shows
# 1e-5 voxel typical, 3e-4 at most, on cone_small).  A_S sums them along
# the ray, where the shifts cancel in pairs (1e-6 relative); A_S^T adds each
# into its own voxel, where they do not, and random data measures 1.1e-5.
SIDDON_T_TOL = 3e-5


@pytest.mark.parametrize("spec", SIDDON_CASES, ids=lambda s: s.name)
def test_siddon_At_matches_oracle(ct, spec):
    g = ct.Geometry.from_spec(spec, projector="siddon")
    y = ci.random_vector(spec.m, seed=74).astype(np.float32).reshape(spec.sino_shape)
    x = host(ct.adjoint_At(g, dev(y)))
    ref = oracle.adjoint_St(spec, y.astype(np.float64))
    assert rel(x, ref) <= SIDDON_T_TOL, rel(x, ref)


def test_siddon_bf16_volume_and_full_size_rays(ct):
    """BF16 storage reads the same walk from the rounded copy; at 256^3 the
    walk is checked on sampled rays against the oracle."""
    spec = ci.CONE_SMALL
    g = ct.Geometry.from_spec(spec, projector="siddon", vol_dtype="bf16")
    x = volume_input(spec, "phantom")
    y = host(ct.project_A(g, dev(x)))
    xr = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert rel(y, oracle.project_S(spec, xr.astype(np.float64))) <= OP_TOL
    spec = ci.CONE_256
    g = ct.Geometry.from_spec(spec, projector="siddon")
    x = ci.phantom(spec)[0]
    y = host(ct.project_A(g, dev(x))).reshape(-1)
    rays = ci.sample_indices(spec.m, 2000, seed=75)
    ref = oracle.project_S_rays(spec, x.astype(np.float64), rays)
    assert rel(y[rays], ref) <= OP_TOL, rel(y[rays], ref)


def test_siddon_gpu_dot_product(ct):
    spec = ci.CONE_ANISO
    g = ct.Geometry.from_spec(spec, projector="siddon")
    x = dev(ci.random_vector(spec.n, seed=76).reshape(spec.vol_shape))
    y = dev(ci.random_vector(spec.m, seed=77).reshape(spec.sino_shape))
    ax = ct.project_A(g, x).double()
    lhs = float((ax * y.double()).sum())
    rhs = float((x.double() * ct.adjoint_At(g, y).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(ax.norm() * y.double().norm())


@pytest.mark.parametrize("spec", ci.DEGENERATE, ids=lambda s: s.name)
def test_degenerate_scans_match_oracle(ct, spec):
    """One voxel, one view, a one-row cone-beam detector, a one-voxel-wide
    column, three detector bins: every operator against the oracle over its
    whole output (tiles far larger than the grid, z runs past nz, lanes past
    nu and nv)."""
    g = ct.Geometry.from_spec(spec)
    x = ci.random_vector(spec.n, seed=71, positive=True).astype(np.float32).reshape(spec.vol_shape)
    y = ci.random_vector(spec.m, seed=72, positive=True).astype(np.float32).reshape(spec.sino_shape)
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    checks = [
        ("A", host(ct.project_A(g, dev(x))), oracle.project_A(spec, x64)),
        ("B_un", host(ct.backproject_B(g, dev(y), "un")), oracle.backproject_B(spec, y64)),
        ("B_fbp", host(ct.backproject_B(g, dev(y), "fbp")), oracle.backproject_B(spec, y64, filtered=True)),
        ("F", host(ct.ramp_F(g, dev(y))), oracle.ramp_F(spec, y64)),
        ("At", host(ct.adjoint_At(g, dev(y))), oracle.adjoint_At(spec, y64)),
        ("Bt_un", host(ct.adjoint_Bt(g, dev(x), "un")), oracle.adjoint_Bt(spec, x64, filtered=False)),
        ("Bt_fbp", host(ct.adjoint_Bt(g, dev(x), "fbp")), oracle.adjoint_Bt(spec, x64, filtered=True)),
    ]
    for name, out, ref in checks:
        assert rel(out, ref) <= OP_TOL, (name, rel(out, ref))


@pytest.mark.parametrize("spec", [s for s in ci.DEGENERATE if s.kind == ci.CONE_3D], ids=lambda s: s.name)
def test_siddon_on_degenerate_scans_matches_oracle(ct, spec):
    """The line-intersection projector and its transpose on the degenerate
    cone-beam scans (a one-voxel grid, one view, one detector row, a
    one-voxel column)."""
    g = ct.Geometry.from_spec(spec, projector="siddon")
    x = ci.random_vector(spec.n, seed=75, positive=True).astype(np.float32).reshape(spec.vol_shape)
    y = ci.random_vector(spec.m, seed=76, positive=True).astype(np.float32).reshape(spec.sino_shape)
    out = host(ct.project_A(g, dev(x)))
    ref = oracle.project_S(spec, x.astype(np.float64))
    assert rel(out, ref) <= OP_TOL, rel(out, ref)
    back = host(ct.adjoint_At(g, dev(y)))
    ref_t = oracle.adjoint_St(spec, y.astype(np.float64))
    assert rel(back, ref_t) <= SIDDON_T_TOL, rel(back, ref_t)


# seed 171: 28 slices of 2.617 mm, whose central detector row lies in a
# slice boundary plane (the positive-side reading)
@pytest.mark.parametrize("seed", list(range(24)) + [171])
def test_random_scans_match_oracle(ct, seed):
    """Seeded random small scans (ct_inputs.random_geometry: grid, views,
    short and full spans, start angle, magnification, detector coverage and
    pixel aspect all drawn): every operator of both projectors against the
    oracle over its whole output."""
    spec = ci.random_geometry(seed)
    g = ct.Geometry.from_spec(spec)
    x = ci.random_vector(spec.n, seed=77, positive=True).astype(np.float32).reshape(spec.vol_shape)
    y = ci.random_vector(spec.m, seed=78, positive=True).astype(np.float32).reshape(spec.sino_shape)
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    checks = [
        ("A", host(ct.project_A(g, dev(x))), oracle.project_A(spec, x64), OP_TOL),
        ("B_un", host(ct.backproject_B(g, dev(y), "un")), oracle.backproject_B(spec, y64), OP_TOL),
        ("B_fbp", host(ct.backproject_B(g, dev(y), "fbp")), oracle.backproject_B(spec, y64, filtered=True), OP_TOL),
        ("F", host(ct.ramp_F(g, dev(y))), oracle.ramp_F(spec, y64), OP_TOL),
        ("At", host(ct.adjoint_At(g, dev(y))), oracle.adjoint_At(spec, y64), OP_TOL),
        ("Bt_un", host(ct.adjoint_Bt(g, dev(x), "un")), oracle.adjoint_Bt(spec, x64, filtered=False), OP_TOL),
        ("Bt_fbp", host(ct.adjoint_Bt(g, dev(x), "fbp")), oracle.adjoint_Bt(spec, x64, filtered=True), OP_TOL),
    ]
    if spec.kind == ci.CONE_3D:
        gs = ct.Geometry.from_spec(spec, projector="siddon")
        checks += [("A_S", host(ct.project_A(gs, dev(x))), oracle.project_S(spec, x64), OP_TOL),
                   ("A_S^T", host(ct.adjoint_At(gs, dev(y))), oracle.adjoint_St(spec, y64), SIDDON_T_TOL)]
    for name, out, ref, tol in checks:
        assert rel(out, ref) <= tol, (spec, name, rel(out, ref))

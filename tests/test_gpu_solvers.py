"""GPU parity of the solvers (BA-GMRES, AB-GMRES, CGLS) and of the Arnoldi
building blocks against the FP64 oracle, through the C-ABI.

Tolerances: the reconstructed image and the residual history after k
iterations agree with the FP64 oracle to relative error <= 1e-4 (residuals
relative to resid[0]), or, where the k-th iterate is more sensitive than
that to FP32 operator error, to 3x the oracle's own sensitivity: the oracle
is run a second time with every operator output perturbed by a seeded
relative error of 1e-6 (the class of the FP32 operators' error, which the
operator tests bound by 1e-5 and measure at ~3e-7 to 7e-7), and its
deviation d_k from the unperturbed run (computed by the oracle alone) is
what an FP32 implementation can be expected to reach at iteration k; near a
stagnation of GMRES on noisy data d_k reaches 1e-2.  Full-size solves are
checked through properties that hold at any size.
"""
import numpy as np
import pytest
import torch

import ct_inputs as ci
import oracle
from oracle import krylov

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-4


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


OP_EPS = 1e-6


def _perturbed(f, rng):
    def g(v):
        y = np.asarray(f(v), dtype=np.float64)
        return y * (1.0 + OP_EPS * rng.standard_normal(y.shape))
    return g


def oracle_with_sensitivity(solver, spec, b_kind, b, k, **kw):
    """FP64 oracle solve, plus the tolerances that an FP32-class operator
    error allows at iteration k (image, residual history)."""
    ops = oracle.Operators(spec, b_kind)
    b64 = b.astype(np.float64).reshape(-1)
    ref = solver(ops.A, ops.B, b64, k, **kw)
    rng = np.random.default_rng(97)
    pert = solver(_perturbed(ops.A, rng), _perturbed(ops.B, rng), b64, k, **kw)
    d_img = rel(pert["x_final"], ref["x_final"])
    key = "data_resid" if kw.get("record_data_resid") else "resid"
    d_res = np.max(np.abs(pert[key] - ref[key])) / ref[key][0]
    return ref, max(SOLVE_TOL, 3 * d_img), max(SOLVE_TOL, 3 * d_res)


def data_for(spec, noise=0.01, seed=81):
    x = ci.phantom(spec)[0].astype(np.float64)
    b = oracle.project_A(spec, x)
    if noise:
        b = b + ci.gaussian_noise(b.shape, noise * b.max(), seed=seed)
    return b.astype(np.float32), x


CASES = [(ci.CONE_SMALL, "un", 20), (ci.CONE_SMALL, "fbp", 12), (ci.CONE_ANISO, "un", 15),
         (ci.PAR2D_64, "un", 30), (ci.PAR2D_ANISO, "fbp", 10), (ci.CONE_512_CUT64, "un", 15)]


@pytest.mark.parametrize("spec,b_kind,k", CASES, ids=lambda v: getattr(v, "name", str(v)))
@pytest.mark.parametrize("dot_mode", [1, 0])
def test_bagmres_matches_oracle(ct, spec, b_kind, k, dot_mode):
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.bagmres(g, dev(b), k, b_kind=b_kind, dot_mode=dot_mode)
    ref, tol_x, tol_r = oracle_with_sensitivity(krylov.ba_gmres, spec, b_kind, b, k, keep_basis=False)
    assert res.iters == k
    assert np.max(np.abs(res.resid - ref["resid"])) <= tol_r * ref["resid"][0]
    assert rel(host(x), ref["x_final"]) <= tol_x, (rel(host(x), ref["x_final"]), tol_x)
    assert np.all(np.diff(res.resid) <= 1e-6 * res.resid[0])


@pytest.mark.parametrize("spec,b_kind,k", [(ci.CONE_SMALL, "un", 12), (ci.PAR2D_64, "un", 20),
                                           (ci.CONE_ANISO, "fbp", 8)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_abgmres_matches_oracle(ct, spec, b_kind, k):
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.abgmres(g, dev(b), k, b_kind=b_kind)
    ref, tol_x, tol_r = oracle_with_sensitivity(krylov.ab_gmres, spec, b_kind, b, k, keep_basis=False)
    assert np.max(np.abs(res.resid - ref["resid"])) <= tol_r * ref["resid"][0]
    assert rel(host(x), ref["x_final"]) <= tol_x, (rel(host(x), ref["x_final"]), tol_x)


@pytest.mark.parametrize("spec,b_kind,k", [(ci.PAR2D_64, "un", 30), (ci.CONE_SMALL, "at", 15),
                                           (ci.CONE_SMALL, "un", 8)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_cgls_matches_oracle(ct, spec, b_kind, k):
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.cgls(g, dev(b), k, b_kind=b_kind)
    ref, tol_x, tol_r = oracle_with_sensitivity(krylov.cgls, spec, b_kind, b, k)
    assert np.max(np.abs(res.resid - ref["resid"])) <= tol_r * ref["resid"][0]
    assert rel(host(x), ref["x_final"]) <= tol_x, (rel(host(x), ref["x_final"]), tol_x)


def test_cgls_record_data_resid(ct):
    spec = ci.CONE_SMALL
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.cgls(g, dev(b), 6, b_kind="un", record_data_resid=True)
    ref, _, tol_r = oracle_with_sensitivity(krylov.cgls, spec, "un", b, 6, record_data_resid=True)
    assert np.max(np.abs(res.resid - ref["data_resid"])) <= tol_r * ref["data_resid"][0]


def test_unmatched_cgls_diverges_on_gpu(ct):
    """Sec. III: CGLS with (A, B_un) reaches a minimum data residual and
    then grows, while BA-GMRES keeps lowering ||BAx - Bb||."""
    spec = ci._cone("tinycone", 8, 10.0, 12, 13, 9, 14.0, ang0=0.2)
    x = ci.random_vector(spec.n, 1, positive=True)
    b = oracle.project_A(spec, x).astype(np.float32)
    g = ct.Geometry.from_spec(spec)
    _, res = ct.cgls(g, dev(b), 50, b_kind="un", record_data_resid=True)
    r = res.resid[:res.iters + 1]
    jmin = int(np.argmin(r))
    assert 0 < jmin < 40 and r[-1] > 10 * r[jmin]
    _, ba = ct.bagmres(g, dev(b), 40)
    assert np.all(np.diff(ba.resid[:ba.iters + 1]) <= 1e-6 * ba.resid[0])


def test_zero_data_is_a_lucky_breakdown(ct):
    spec = ci.CONE_ANISO
    g = ct.Geometry.from_spec(spec)
    x = torch.full(spec.vol_shape, 7.0, device="cuda")
    res = ct.ct_bagmres_solve(g, torch.zeros(spec.sino_shape, device="cuda"), 5, x)
    assert res.status == ct.CT_BREAKDOWN_LUCKY and res.iters == 0
    assert torch.count_nonzero(x) == 0
    assert res.resid[0] == 0.0 and np.all(res.resid[1:] == -1.0)


def test_full_dimension_reaches_exact_solution(ct):
    """Consistent data for a 2D problem with n = 4 unknowns: after n
    iterations the Krylov space is the whole space and BA-GMRES returns the
    exact solution of BAx = Bb, here x_true."""
    spec = ci.Geometry("n4", ci.PARALLEL_2D, 2, 2, 1, 1.0, 6, 0.0, np.pi, 5, 1, 1.0, 1.0)
    xt = np.array([1.0, 2.0, 0.5, 3.0])
    b = oracle.project_A(spec, xt).astype(np.float32)
    g = ct.Geometry.from_spec(spec)
    x = torch.empty(spec.vol_shape, device="cuda")
    res = ct.ct_bagmres_solve(g, dev(b), 4, x)
    assert res.iters == 4
    assert res.status in (ct.CT_BREAKDOWN_LUCKY, ct.CT_OK)
    assert rel(host(x), xt) < 1e-4
    assert res.resid[4] <= 1e-5 * res.resid[0]


def test_tolerance_stop(ct):
    spec = ci.CONE_SMALL
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.bagmres(g, dev(b), 30, tol=0.05)
    assert 0 < res.iters < 30
    assert res.resid[res.iters] <= 0.05 * res.resid[0] < res.resid[res.iters - 1]
    assert np.all(res.resid[res.iters + 1:] == -1.0)
    x2, res2 = ct.bagmres(g, dev(b), res.iters)
    assert torch.equal(x, x2)


def test_workspace_and_determinism(ct):
    spec = ci.CONE_SMALL
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    bd = dev(b)
    x1 = torch.empty(spec.vol_shape, device="cuda")
    x2 = torch.empty(spec.vol_shape, device="cuda")
    r1 = ct.ct_bagmres_solve(g, bd, 10, x1, ct.make_opts(b_kind="fbp"), workspace="torch")
    r2 = ct.ct_bagmres_solve(g, bd, 10, x2, ct.make_opts(b_kind="fbp"), workspace=None)
    assert torch.equal(x1, x2) and np.array_equal(r1.resid, r2.resid)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(ct.CTError) as ei:
        ct.ct_bagmres_solve(g, bd, 10, x1, ct.make_opts(workspace=small), workspace=None)
    assert ei.value.status == ct.CT_ENOMEM


def test_host_buffer_solve_equals_device_solve(ct):
    """ct_bagmres_solve_host (b and x in pinned host memory, copies inside
    the call) runs the same kernels as the device-buffer solve: identical
    image and residual history."""
    spec = ci.CONE_ANISO
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    xd = torch.empty(spec.vol_shape, device="cuda")
    rd = ct.ct_bagmres_solve(g, dev(b), 8, xd, ct.make_opts(b_kind="fbp"))
    bh = torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32)).pin_memory()
    xh = torch.full(spec.vol_shape, float("nan")).pin_memory()
    rh = ct.ct_bagmres_solve_host(g, bh, 8, xh, ct.make_opts(b_kind="fbp"))
    assert rh.iters == rd.iters == 8
    assert torch.equal(xh, xd.cpu()) and np.array_equal(rh.resid, rd.resid)
    with pytest.raises(TypeError):
        ct.ct_bagmres_solve_host(g, dev(b), 8, xh)


def test_reorthogonalisation_keeps_parity(ct):
    spec = ci.CONE_SMALL
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.bagmres(g, dev(b), 20, reorth=1)
    ref, tol_x, tol_r = oracle_with_sensitivity(krylov.ba_gmres, spec, "un", b, 20, keep_basis=False)
    assert rel(host(x), ref["x_final"]) <= tol_x
    assert np.max(np.abs(res.resid - ref["resid"])) <= tol_r * ref["resid"][0]


@pytest.mark.parametrize("dot_mode", [0, 1])
@pytest.mark.parametrize("length", [1, 1000, 1 << 20, (1 << 20) + 3])
def test_mgs_sweep_against_definition(ct, dot_mode, length):
    """One MGS sweep equals the textbook recurrence h_i = <q, v_i>,
    q -= h_i v_i (FP64 numpy), then h_j = ||q||."""
    j = 6
    rng = np.random.default_rng(90 + length % 7)
    Q, _ = np.linalg.qr(rng.standard_normal((length, j))) if length >= j else (
        rng.standard_normal((length, j)), None)
    ldv = length + (64 - length % 64) % 64
    V = np.zeros((j, ldv), dtype=np.float32)
    V[:, :length] = Q.T.astype(np.float32)
    q0 = rng.standard_normal(length).astype(np.float32) + 0.5 * V[0, :length]
    qd = dev(q0)
    h = torch.zeros(j + 1, dtype=torch.float64, device="cuda")
    ct.ct_mgs_sweep(dev(V), ldv, j, length, qd, h, dot_mode)
    q = q0.astype(np.float64).copy()
    href = np.zeros(j + 1)
    for i in range(j):
        href[i] = q @ V[i, :length].astype(np.float64)
        q -= href[i] * V[i, :length].astype(np.float64)
    href[j] = np.linalg.norm(q)
    hg = host(h)
    assert np.max(np.abs(hg - href)) <= 1e-5 * np.linalg.norm(q0)
    assert rel(host(qd), q) <= 1e-5


def test_basis_combine_against_definition(ct):
    k, length = 9, 123457
    rng = np.random.default_rng(95)
    ldv = length + 11
    V = rng.standard_normal((k, ldv)).astype(np.float32)
    y = rng.standard_normal(k)
    x = torch.empty(length, device="cuda")
    ct.ct_basis_combine(dev(V), ldv, k, length, torch.from_numpy(y).cuda(), x)
    ref = (y[:, None] * V[:, :length].astype(np.float64)).sum(axis=0)
    assert rel(host(x), ref) <= 1e-6


@pytest.mark.parametrize("b_kind,k", [("fbp", 40), ("un", 20)])
def test_full_size_256_bagmres_properties(ct, b_kind, k):
    """The 256^3 headline solve (Poisson data): the residual history is
    non-increasing, its last entry matches the recomputed ||B(b - A x_k)||,
    and the first iterations agree with the oracle's closed forms: resid[0]
    = ||B b|| and resid[1] = min_c ||B b - c B A B b|| (one-dimensional
    least squares)."""
    spec = ci.CONE_256
    g = ct.Geometry.from_spec(spec)
    x_true = ci.phantom(spec)[0]
    p = host(ct.project_A(g, dev(x_true)))
    b = dev(ci.poisson_log_data(p, seed=1))
    x, res = ct.bagmres(g, b, k, b_kind=b_kind)
    r = res.resid
    assert res.iters == k
    assert np.all(np.diff(r) <= 1e-6 * r[0])
    Bb = ct.backproject_B(g, b, b_kind).double()
    true = float(torch.linalg.vector_norm(Bb - ct.backproject_B(g, ct.project_A(g, x), b_kind).double()))
    assert abs(true - r[-1]) <= 2e-3 * r[0], (true, r[-1])
    assert abs(float(torch.linalg.vector_norm(Bb)) - r[0]) <= 1e-6 * r[0]
    s1 = ct.backproject_B(g, ct.project_A(g, Bb.float()), b_kind).double()
    c = float((s1 * Bb).sum() / (s1 * s1).sum())
    r1 = float(torch.linalg.vector_norm(Bb - c * s1))
    assert abs(r1 - r[1]) <= 1e-4 * r[0], (r1, r[1])


def test_error_history_matches_oracle(ct):
    """ct_bagmres_solve_err: err[j] = ||x_j - x_true|| of every iterate (the
    semi-convergence curve, Sec. III Fig. 4) against the FP64 oracle's
    iterates, each within max(1e-4 ||x_j||, 3 d_j), d_j the distance between
    the oracle's iterate and its own run with FP32-class (1e-6) operator
    error; x_out is the plain solve's x_k."""
    spec, k = ci.CONE_SMALL, 12
    b, x_true = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x = torch.empty(spec.vol_shape, device="cuda")
    res, err = ct.ct_bagmres_solve_err(g, dev(b), k, x, dev(x_true), ct.make_opts(b_kind="fbp"))
    x_plain = torch.empty_like(x)
    res_plain = ct.ct_bagmres_solve(g, dev(b), k, x_plain, ct.make_opts(b_kind="fbp"))
    assert torch.equal(x, x_plain) and np.array_equal(res.resid, res_plain.resid)
    ops = oracle.Operators(spec, "fbp")
    b64 = b.astype(np.float64).reshape(-1)
    ref = krylov.ba_gmres(ops.A, ops.B, b64, k, keep_basis=False)
    rng = np.random.default_rng(97)
    pert = krylov.ba_gmres(_perturbed(ops.A, rng), _perturbed(ops.B, rng), b64, k, keep_basis=False)
    xt = x_true.reshape(-1)
    assert abs(err[0] - np.linalg.norm(xt)) <= 1e-5 * np.linalg.norm(xt)
    for j in range(1, k + 1):
        xj = ref["x"][j - 1]
        tol = max(SOLVE_TOL * np.linalg.norm(xj), 3 * np.linalg.norm(pert["x"][j - 1] - xj))
        assert abs(err[j] - np.linalg.norm(xj - xt)) <= tol, (j, err[j], np.linalg.norm(xj - xt), tol)


def test_error_history_marks_iterations_not_done(ct):
    spec = ci.CONE_ANISO
    b, x_true = data_for(spec, noise=0.0)
    g = ct.Geometry.from_spec(spec)
    x = torch.empty(spec.vol_shape, device="cuda")
    res, err = ct.ct_bagmres_solve_err(g, dev(b), 30, x, dev(x_true), ct.make_opts(b_kind="fbp", tol=1e-2))
    assert 0 < res.iters < 30
    assert np.all(err[res.iters + 1:] == -1.0) and np.all(err[:res.iters + 1] >= 0.0)


@pytest.mark.parametrize("spec,b_kind", [(ci.CONE_SMALL, "un"), (ci.PAR2D_64, "fbp")],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_restarted_matches_oracle(ct, spec, b_kind):
    """ct_bagmres_restarted, 3 cycles of GMRES(5), against the FP64 oracle's
    restarted solve (same tolerance rule as the unrestarted solves)."""
    m, cycles = 5, 3
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x = torch.empty(spec.vol_shape, device="cuda")
    res = ct.ct_bagmres_restarted(g, dev(b), m, cycles, x, ct.make_opts(b_kind=b_kind))
    ref, tol_x, tol_r = oracle_with_sensitivity(
        lambda A, B, bb, k: krylov.ba_gmres_restarted(A, B, bb, m, cycles), spec, b_kind, b, m * cycles)
    assert res.iters == m * cycles
    assert np.max(np.abs(res.resid - ref["resid"])) <= tol_r * ref["resid"][0]
    assert rel(host(x), ref["x_final"]) <= tol_x, (rel(host(x), ref["x_final"]), tol_x)
    assert np.all(np.diff(res.resid) <= 1e-6 * res.resid[0])


def test_restarted_single_cycle_equals_solve(ct):
    spec = ci.CONE_ANISO
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x1 = torch.empty(spec.vol_shape, device="cuda")
    x2 = torch.empty(spec.vol_shape, device="cuda")
    r1 = ct.ct_bagmres_solve(g, dev(b), 7, x1, ct.make_opts(b_kind="un"))
    r2 = ct.ct_bagmres_restarted(g, dev(b), 7, 1, x2, ct.make_opts(b_kind="un"))
    assert torch.equal(x1, x2) and np.array_equal(r1.resid, r2.resid)
    with pytest.raises(ct.CTError):
        ct.ct_bagmres_restarted(g, dev(b), 7, 0, x2)


@pytest.mark.parametrize("spec,b_kind,k", [(ci.CONE_SMALL, "un", 12), (ci.PAR2D_64, "fbp", 15)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_bagmres_with_siddon_projector_matches_oracle(ct, spec, b_kind, k):
    """BA-GMRES with the line-intersection A and the same unmatched B."""
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec, projector="siddon")
    x = torch.empty(spec.vol_shape, device="cuda")
    res = ct.ct_bagmres_solve(g, dev(b), k, x, ct.make_opts(b_kind=b_kind))
    ops = oracle.Operators(spec, b_kind, projector="siddon")
    b64 = b.astype(np.float64).reshape(-1)
    ref = krylov.ba_gmres(ops.A, ops.B, b64, k, keep_basis=False)
    rng = np.random.default_rng(97)
    pert = krylov.ba_gmres(_perturbed(ops.A, rng), _perturbed(ops.B, rng), b64, k, keep_basis=False)
    tol_x = max(SOLVE_TOL, 3 * rel(pert["x_final"], ref["x_final"]))
    tol_r = max(SOLVE_TOL, 3 * np.max(np.abs(pert["resid"] - ref["resid"])) / ref["resid"][0])
    assert np.max(np.abs(res.resid - ref["resid"])) <= tol_r * ref["resid"][0]
    assert rel(host(x), ref["x_final"]) <= tol_x, (rel(host(x), ref["x_final"]), tol_x)

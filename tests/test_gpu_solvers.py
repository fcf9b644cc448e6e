"""GPU parity of the solvers (BA-GMRES, AB-GMRES, CGLS) and of the Arnoldi
building blocks against the FP64 oracle, through the C-ABI.

Tolerances: the reconstructed image and the residual history after k
iterations agree with the FP64 oracle to relative error <= 1e-4 (residuals
relative to resid[0]).  The cases listed in EXCEPTIONS are held instead to
3x the oracle's own sensitivity: the oracle is run a second time with every
operator output perturbed by a seeded relative error of 1e-6 (the class of
the FP32 operators' error, which the operator tests bound by 1e-5 and
measure at ~3e-7 to 7e-7), and its deviation d_k from the unperturbed run
(computed by the oracle alone) is what an FP32 implementation can be
expected to reach at iteration k.  Each exception records its measured d_k
and GPU error, and whether a variant of the solver (plain FP32 dot
products, a second MGS sweep) meets the flat bar; where one does, that
variant is held to 1e-4 in the same test.  Full-size solves are
checked through properties that hold at any size, and against the oracle's
stored solves in tests/test_gpu_large.py.

Every parity case records, through the ``parity_log`` fixture (a JSON line
per case when CT_PARITY_REPORT names a file): k, d_img and d_res, the
tolerances in force and the GPU's errors.  Where a GPU error is above the
flat 1e-4, the case also records the errors of the solve rerun with plain
FP32 dot products (dot_mode = 1) and with a second MGS sweep (reorth = 1).
"""
import numpy as np
import pytest
import torch

import ct_inputs as ci
import oracle
from oracle import krylov

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-4

# (solver, scan, b_kind, k, dot_mode) -> why the k-th iterate is held to 3 d_k
# rather than 1e-4 (measured on a GB300: d = the oracle's sensitivity to a
# 1e-6 operator perturbation, err = the GPU's distance to the oracle), and
# the solver variant, if any, that meets 1e-4 on the same case.
EXCEPTIONS = {
    ("ba", "par2d_64", "un", 30, 0): dict(
        why="noisy 2D scan, 30 iterations past the semi-convergence minimum: d_img = 5.9e-4, "
            "GPU image error 1.1e-4 with compensated dots and one MGS sweep",
        flat_with="reorth=1"),   # measured 4.4e-5 with the second sweep
    ("ab", "par2d_64", "un", 20, 0): dict(
        why="AB-GMRES image x = B y_20 on the noisy 2D scan: d_img = 8.9e-3, GPU image error 8.9e-3 "
            "(the same with plain dots or a second sweep, 8.9e-3); residual history within 1e-4",
        flat_with=None),
}


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


class Sensitive:
    """An FP64 oracle solve with its sensitivity: ``ref`` the oracle's
    result, ``d_img`` = ||x_pert - x|| / ||x|| and ``d_res`` =
    max_j |r_pert[j] - r[j]| / r[0] for the oracle rerun with FP32-class
    (1e-6) operator error; ``sens_x``, ``sens_r`` = max(1e-4, 3 d), the
    tolerances of a listed exception."""

    def __init__(self, ref, d_img, d_res, key="resid"):
        self.ref, self.d_img, self.d_res, self.key = ref, float(d_img), float(d_res), key
        self.sens_x = max(SOLVE_TOL, 3 * self.d_img)
        self.sens_r = max(SOLVE_TOL, 3 * self.d_res)

    def errors(self, x_gpu, resid_gpu):
        r = self.ref[self.key]
        return rel(x_gpu, self.ref["x_final"]), float(np.max(np.abs(np.asarray(resid_gpu) - r)) / r[0])

    def check(self, parity_log, k, x_gpu, resid_gpu, rerun=None, solver="ba", case="", b_kind="un",
              dot_mode=0, **info):
        """Logs the case and asserts the GPU result is within tolerance:
        1e-4, or 3 d_k for a listed exception.  ``rerun(**opts)`` -> (x,
        resid) reruns the GPU solve with other options; it is called when an
        error exceeds 1e-4 (for the record, and for an exception's variant
        that must meet 1e-4)."""
        exc = EXCEPTIONS.get((solver, case, b_kind, k, dot_mode))
        tol_x = self.sens_x if exc else SOLVE_TOL
        tol_r = self.sens_r if exc else SOLVE_TOL
        err_img, err_res = self.errors(x_gpu, resid_gpu)
        variants = {}
        if rerun is not None and max(err_img, err_res) > SOLVE_TOL:
            for name, opts in (("dot_mode=1", dict(dot_mode=1)), ("reorth=1", dict(reorth=1))):
                e = self.errors(*rerun(**opts))
                variants[name] = {"err_img": e[0], "err_res": e[1]}
        parity_log(k=k, d_img=self.d_img, d_res=self.d_res, tol_x=tol_x, tol_r=tol_r, err_img=err_img,
                   err_res=err_res, variants=variants, exception=bool(exc), solver=solver, case=case,
                   b_kind=b_kind, dot_mode=dot_mode, **info)
        assert err_res <= tol_r, ("residual history", err_res, tol_r)
        assert err_img <= tol_x, ("image", err_img, tol_x)
        if exc and exc["flat_with"] and max(err_img, err_res) > SOLVE_TOL:
            v = variants[exc["flat_with"]]
            assert v["err_img"] <= SOLVE_TOL and v["err_res"] <= SOLVE_TOL, (exc["flat_with"], v)


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
    return Sensitive(ref, d_img, d_res, key)


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
def test_bagmres_matches_oracle(ct, parity_log, spec, b_kind, k, dot_mode):
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.bagmres(g, dev(b), k, b_kind=b_kind, dot_mode=dot_mode)
    sens = oracle_with_sensitivity(krylov.ba_gmres, spec, b_kind, b, k, keep_basis=False)
    assert res.iters == k
    assert np.all(np.diff(res.resid) <= 1e-6 * res.resid[0])

    def rerun(**o):
        o.setdefault("dot_mode", dot_mode)
        xx, rr = ct.bagmres(g, dev(b), k, b_kind=b_kind, **o)
        return host(xx), rr.resid
    sens.check(parity_log, k, host(x), res.resid, rerun, solver="ba", case=spec.name, b_kind=b_kind,
               dot_mode=dot_mode)


@pytest.mark.parametrize("spec,b_kind,k", [(ci.CONE_SMALL, "un", 12), (ci.PAR2D_64, "un", 20),
                                           (ci.CONE_ANISO, "fbp", 8)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_abgmres_matches_oracle(ct, parity_log, spec, b_kind, k):
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.abgmres(g, dev(b), k, b_kind=b_kind)
    sens = oracle_with_sensitivity(krylov.ab_gmres, spec, b_kind, b, k, keep_basis=False)

    def rerun(**o):
        xx, rr = ct.abgmres(g, dev(b), k, b_kind=b_kind, **o)
        return host(xx), rr.resid
    sens.check(parity_log, k, host(x), res.resid, rerun, solver="ab", case=spec.name, b_kind=b_kind)


@pytest.mark.parametrize("spec,b_kind,k", [(ci.PAR2D_64, "un", 30), (ci.CONE_SMALL, "at", 15),
                                           (ci.CONE_SMALL, "un", 8)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_cgls_matches_oracle(ct, parity_log, spec, b_kind, k):
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.cgls(g, dev(b), k, b_kind=b_kind)
    sens = oracle_with_sensitivity(krylov.cgls, spec, b_kind, b, k)
    sens.check(parity_log, k, host(x), res.resid, solver="cgls", case=spec.name, b_kind=b_kind)


def test_cgls_record_data_resid(ct, parity_log):
    spec = ci.CONE_SMALL
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.cgls(g, dev(b), 6, b_kind="un", record_data_resid=True)
    sens = oracle_with_sensitivity(krylov.cgls, spec, "un", b, 6, record_data_resid=True)
    sens.check(parity_log, 6, host(x), res.resid, solver="cgls", case=spec.name, b_kind="un",
               record_data_resid=True)


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


def test_reorthogonalisation_keeps_parity(ct, parity_log):
    spec = ci.CONE_SMALL
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.bagmres(g, dev(b), 20, reorth=1)
    sens = oracle_with_sensitivity(krylov.ba_gmres, spec, "un", b, 20, keep_basis=False)
    sens.check(parity_log, 20, host(x), res.resid, solver="ba", case=spec.name, b_kind="un", reorth=1)


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


def test_error_history_matches_oracle(ct, parity_log):
    """ct_bagmres_solve_err: err[j] = ||x_j - x_true|| of every iterate (the
    semi-convergence curve, Sec. III Fig. 4) against the FP64 oracle's
    iterates, each within 1e-4 ||x_j|| (the image bar); x_out is the plain
    solve's x_k."""
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
    worst = 0.0
    for j in range(1, k + 1):
        xj = ref["x"][j - 1]
        assert abs(err[j] - np.linalg.norm(xj - xt)) <= SOLVE_TOL * np.linalg.norm(xj), \
            (j, err[j], np.linalg.norm(xj - xt))
        worst = max(worst, abs(err[j] - np.linalg.norm(xj - xt)) / np.linalg.norm(xj))
    d = max(np.linalg.norm(pert["x"][j - 1] - ref["x"][j - 1]) / np.linalg.norm(ref["x"][j - 1])
            for j in range(1, k + 1))
    parity_log(k=k, d_img=d, err_img=worst, tol_x=SOLVE_TOL, solver="ba_err_hist", case=spec.name, b_kind="fbp")


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
def test_restarted_matches_oracle(ct, parity_log, spec, b_kind):
    """ct_bagmres_restarted, 3 cycles of GMRES(5), against the FP64 oracle's
    restarted solve (same tolerance rule as the unrestarted solves)."""
    m, cycles = 5, 3
    b, _ = data_for(spec)
    g = ct.Geometry.from_spec(spec)
    x = torch.empty(spec.vol_shape, device="cuda")
    res = ct.ct_bagmres_restarted(g, dev(b), m, cycles, x, ct.make_opts(b_kind=b_kind))
    sens = oracle_with_sensitivity(
        lambda A, B, bb, k: krylov.ba_gmres_restarted(A, B, bb, m, cycles), spec, b_kind, b, m * cycles)
    assert res.iters == m * cycles
    assert np.all(np.diff(res.resid) <= 1e-6 * res.resid[0])
    sens.check(parity_log, m * cycles, host(x), res.resid, solver="ba_restarted", case=spec.name,
               b_kind=b_kind)


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
def test_bagmres_with_siddon_projector_matches_oracle(ct, parity_log, spec, b_kind, k):
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
    sens = Sensitive(ref, rel(pert["x_final"], ref["x_final"]),
                     np.max(np.abs(pert["resid"] - ref["resid"])) / ref["resid"][0])

    def rerun(**o):
        xx = torch.empty(spec.vol_shape, device="cuda")
        rr = ct.ct_bagmres_solve(g, dev(b), k, xx, ct.make_opts(b_kind=b_kind, **o))
        return host(xx), rr.resid
    sens.check(parity_log, k, host(x), res.resid, rerun, solver="ba_siddon", case=spec.name, b_kind=b_kind)


@pytest.mark.parametrize("spec,b_kind,k", [(ci.CONE_1VIEW, "un", 6), (ci.CONE_1ROW, "fbp", 6),
                                          (ci.CONE_COLUMN, "un", 5), (ci.PAR2D_3BIN, "un", 4)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_bagmres_on_degenerate_scans_matches_oracle(ct, parity_log, spec, b_kind, k):
    """BA-GMRES (Eq. 5) on the degenerate scans against the oracle."""
    b = ci.random_vector(spec.m, seed=73, positive=True).astype(np.float32)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.bagmres(g, dev(b.reshape(spec.sino_shape)), k, b_kind=b_kind)
    sens = oracle_with_sensitivity(krylov.ba_gmres, spec, b_kind, b, k, keep_basis=False)
    assert res.status in (ct.CT_OK, ct.CT_BREAKDOWN_LUCKY)
    assert res.iters == len(sens.ref["resid"]) - 1
    sens.check(parity_log, k, host(x), res.resid[:res.iters + 1], case=spec.name, b_kind=b_kind)


def test_one_voxel_scan_breaks_down_after_one_iteration(ct):
    """n = 1: the Krylov space of BA is one-dimensional, so the first
    iteration solves the least-squares problem exactly and reports a lucky
    breakdown; x equals the oracle's (B b) / (B A e) for the single voxel."""
    spec = ci.CONE_VOXEL1
    b = ci.random_vector(spec.m, seed=74, positive=True).astype(np.float32)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.bagmres(g, dev(b.reshape(spec.sino_shape)), 3)
    assert res.status == ct.CT_BREAKDOWN_LUCKY and res.iters == 1
    ops = oracle.Operators(spec, "un")
    bb = float(ops.B(b.astype(np.float64))[0])
    ba = float(ops.B(ops.A(np.ones(1)))[0])
    assert abs(float(host(x)[0, 0, 0]) - bb / ba) <= 1e-5 * abs(bb / ba)


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5, 7, 11])
@pytest.mark.parametrize("solver", ["ba", "ab", "cgls"])
def test_solvers_on_random_scans_match_oracle(ct, parity_log, seed, solver):
    """BA-GMRES (Eq. 5), AB-GMRES (Eq. 4) and CGLS (Eqs. 2-3) on seeded
    random small scans (ct_inputs.random_geometry), 6 iterations, B_FBP for
    the GMRES solves and B_un for CGLS, against the oracle under the solver
    bar."""
    spec = ci.random_geometry(seed)
    k = 6
    b = ci.random_vector(spec.m, seed=79, positive=True).astype(np.float32)
    g = ct.Geometry.from_spec(spec)
    b_kind = "un" if solver == "cgls" else "fbp"
    run = {"ba": ct.bagmres, "ab": ct.abgmres, "cgls": ct.cgls}[solver]
    ref_solver = {"ba": krylov.ba_gmres, "ab": krylov.ab_gmres, "cgls": krylov.cgls}[solver]
    x, res = run(g, dev(b.reshape(spec.sino_shape)), k, b_kind=b_kind)
    kw = {} if solver == "cgls" else {"keep_basis": False}
    sens = oracle_with_sensitivity(ref_solver, spec, b_kind, b, k, **kw)
    n_ref = len(sens.ref["resid"]) - 1
    assert res.iters == n_ref, (res.iters, n_ref)
    if sens.ref["resid"][0] == 0.0:
        # B b = 0 (every voxel centre of a thin-detector scan projects off the
        # detector, so the voxel-driven B sees nothing): x = 0 at once
        assert res.resid[0] == 0.0 and not host(x).any()
        return

    def rerun(**o):
        xx, rr = run(g, dev(b.reshape(spec.sino_shape)), k, b_kind=b_kind, **o)
        return host(xx), rr.resid[:n_ref + 1]
    sens.check(parity_log, k, host(x), res.resid[:n_ref + 1], None if solver == "cgls" else rerun,
               solver=solver, case=spec.name, b_kind=b_kind)


def test_singular_breakdown_keeps_the_residual(ct):
    """AB-GMRES on a scan whose voxel-driven B sees nothing (every voxel
    centre of the 26 slices projects off the 13-row detector, so A B = 0):
    the first iteration breaks down on a zero Hessenberg column, the
    residual stays ||b|| (the oracle's least-squares residual) and x = 0."""
    spec = ci.random_geometry(7)
    b = ci.random_vector(spec.m, seed=79, positive=True).astype(np.float32)
    g = ct.Geometry.from_spec(spec)
    x, res = ct.abgmres(g, dev(b.reshape(spec.sino_shape)), 5, b_kind="fbp")
    ops = oracle.Operators(spec, "fbp")
    ref = krylov.ab_gmres(ops.A, ops.B, b.astype(np.float64), 5, keep_basis=False)
    assert res.status == ct.CT_BREAKDOWN_LUCKY and res.iters == 1 == ref["iters"]
    bn = float(np.linalg.norm(b.astype(np.float64)))
    np.testing.assert_allclose(res.resid[:2], [bn, bn], rtol=1e-6)
    np.testing.assert_allclose(ref["resid"], [bn, bn], rtol=1e-12)
    assert not host(x).any()

"""Differentiation through the C-ABI: autograd for A (backward = exact A^T)
and for the converged BA-GMRES solve x = (BA)^{-1} B b (backward = GMRES on
A^T B^T, then B^T).

* A: torch autograd gradient of <A x, w> equals the oracle's A^T w.
* VJP: the same k adjoint GMRES iterations on the GPU and in the oracle.
* Loss L = ||x - x_ref||^2 for a converged solve (relative residual 1e-6)
  of noiseless data b = A x_true with the ramp-preconditioned B; x_ref is a
  seeded smooth volume, so that dL/dx = 2 (x - x_ref) does not vanish at the
  solution x ~ x_true of the consistent system.
* The 32^3 scan: the GPU gradient dL/db equals the FP64 oracle gradient (the
  oracle's forward and adjoint solves run to 1e-9).  Tolerance max(1e-4, 3 d),
  d = the deviation of the oracle's own gradient when every operator output
  carries a seeded relative error of 1e-6 (the FP32 operators' error class)
  and its solves stop at 1e-6 (computed by the oracle alone).
* The 128^3 scan: central finite differences of L along a seeded smooth
  direction in data space (the projection of a seeded smooth volume) equal
  <dL/db, direction>.  The converged solve is linear in b, so L is quadratic
  and the central difference is exact for any step; a step of half the
  data's norm keeps the FP32 solves' stopping error small against the
  difference, and a smooth direction keeps the perturbed solves as easy as
  the unperturbed one (impulses on single sinogram entries are not: they
  need hundreds more iterations to reach 1e-6).  Every entry of dL/db is
  compared with the FP64 oracle in the 32^3 test.
"""
import numpy as np
import pytest
import torch

import ct_inputs as ci
import oracle
from oracle import krylov

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_07408_gb300 import ct as _ct
    return _ct


@pytest.fixture(scope="module")
def ag(ct):
    from paper_2201_07408_gb300 import autograd
    return autograd


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_project_A_autograd_is_exact_adjoint(ct, ag):
    spec = ci.CONE_ANISO
    g = ct.Geometry.from_spec(spec)
    x = torch.from_numpy(ci.random_vector(spec.n, 1).astype(np.float32).reshape(spec.vol_shape)).cuda()
    w = ci.random_vector(spec.m, 2).astype(np.float32).reshape(spec.sino_shape)
    x.requires_grad_(True)
    y = ag.project_A(g, x)
    (y * torch.from_numpy(w).cuda()).sum().backward()
    ref = oracle.adjoint_At(spec, w.astype(np.float64))
    assert rel(x.grad.cpu().double().numpy(), ref) <= 1e-5


def _consistent_data(spec):
    x_true = ci.phantom(spec)[0].astype(np.float64)
    b = oracle.project_A(spec, x_true).astype(np.float32)
    x_ref = ci.smooth_volume(spec, seed=3) * float(x_true.max())
    return b, x_ref


@pytest.mark.parametrize("b_kind", ["un", "fbp"])
def test_vjp_matches_oracle_vjp(ct, b_kind):
    """The same k adjoint GMRES iterations on the GPU and in the oracle."""
    spec = ci.CONE_GRAD32
    g = ct.Geometry.from_spec(spec)
    gx = ci.random_vector(spec.n, 5).astype(np.float32)
    k = 25
    gb = torch.empty(spec.sino_shape, device="cuda")
    res = ct.ct_bagmres_vjp(g, torch.from_numpy(gx.reshape(spec.vol_shape)).cuda(), k, gb,
                            ct.make_opts(b_kind=b_kind))
    adj = oracle.AdjointOperators(spec, b_kind)
    ref = krylov.ba_gmres_vjp(adj.At, adj.Bt, gx.astype(np.float64), k)
    assert res.iters == k
    assert np.max(np.abs(res.resid - ref["resid"])) <= 1e-4 * ref["resid"][0]
    assert rel(gb.cpu().numpy(), ref["gb"]) <= 1e-4, rel(gb.cpu().numpy(), ref["gb"])


def test_full_gradient_matches_fp64_oracle_32(ct, ag):
    spec = ci.CONE_GRAD32
    b, x_ref = _consistent_data(spec)
    g = ct.Geometry.from_spec(spec)
    tol, kmax = 1e-6, 300
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = ag.bagmres_solve(g, bt, k=kmax, b_kind="fbp", tol=tol)
    loss = ((x.double() - torch.from_numpy(x_ref).cuda()) ** 2).sum()
    loss.backward()
    gb = bt.grad.cpu().double().numpy().reshape(-1)

    ops = oracle.Operators(spec, "fbp")
    adj = oracle.AdjointOperators(spec, "fbp")
    b64 = b.astype(np.float64).reshape(-1)

    def perturbed(f, rng, eps):
        def h(v):
            y = np.asarray(f(v), dtype=np.float64)
            return y * (1.0 + eps * rng.standard_normal(y.shape)) if eps else y
        return h

    def oracle_grad(rtol, eps, kcap):
        rng = np.random.default_rng(99)
        A, B = perturbed(ops.A, rng, eps), perturbed(ops.B, rng, eps)
        At, Bt = perturbed(adj.At, rng, eps), perturbed(adj.Bt, rng, eps)
        fw = krylov.ba_gmres(A, B, b64, kcap, keep_basis=False)
        j = next((i for i, r in enumerate(fw["resid"]) if r <= rtol * fw["resid"][0]), len(fw["x"]))
        xk = fw["x"][max(j, 1) - 1]
        gx = 2.0 * (xk - x_ref.reshape(-1))
        bw = krylov.ba_gmres_vjp(At, Bt, gx, kcap)
        jb = next((i for i, r in enumerate(bw["resid"]) if r <= rtol * bw["resid"][0]), bw["iters"])
        return krylov.ba_gmres_vjp(At, Bt, gx, max(jb, 1))["gb"]

    g_conv = oracle_grad(1e-9, 0.0, 400)
    g_fp32 = oracle_grad(tol, 1e-6, kmax)
    d = rel(g_fp32, g_conv)
    err = rel(gb, g_conv)
    assert err <= max(1e-4, 3 * d), (err, d)


def test_central_differences_128(ct, ag):
    spec = ci.CONE_128
    b, x_ref = _consistent_data(spec)
    xr = torch.from_numpy(x_ref).cuda()
    g = ct.Geometry.from_spec(spec)
    kmax, tol = 300, 1e-6
    bt = torch.from_numpy(b).cuda().requires_grad_(True)
    x = ag.bagmres_solve(g, bt, k=kmax, b_kind="fbp", tol=tol)
    ((x.double() - xr) ** 2).sum().backward()
    gb = bt.grad.reshape(-1).double()

    dx = torch.from_numpy(ci.smooth_volume(spec, seed=8).astype(np.float32)).cuda()
    direction = ct.project_A(g, dx).reshape(-1).double()
    flat = torch.from_numpy(b).cuda().reshape(-1).double()
    h = 0.5 * float(flat.norm() / direction.norm())

    def L(bb):
        xx, res = ct.bagmres(g, bb.float().reshape(spec.sino_shape).contiguous(), kmax, b_kind="fbp", tol=tol)
        # the FP32 residual estimate stalls near 2e-6 on some right-hand sides
        assert res.resid[res.iters] <= 5 * tol * res.resid[0]
        return float(((xx.double() - xr) ** 2).sum())

    fd = (L(flat + h * direction) - L(flat - h * direction)) / (2 * h)
    adj = float((gb * direction).sum())
    assert abs(fd - adj) <= 1e-3 * abs(adj), (fd, adj)

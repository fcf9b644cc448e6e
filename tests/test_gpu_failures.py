"""Failure detection of the solvers, made on the host (no GPU fault).

* A NaN in the data that the caller hands over (host buffers, through
  ct_bagmres_solve_host) makes ||B b|| non-finite: the solve stops before
  its first iteration with CT_ENONFINITE, iters_done = 0 and the history
  marked -1 after resid[0].
* The library's host-side fault injection (ct_fault_set, or CT_FAULT in
  the environment) writes a NaN, an ordinary value, into the new vector of
  iteration N: BA-GMRES, AB-GMRES, the adjoint GMRES of the gradient and
  CGLS stop with CT_ENONFINITE after N - 1 iterations, with the history of
  those iterations equal to an unfaulted run's and -1 after.
* "oom" refuses stream-ordered allocations as if the allocator had failed:
  CT_ENOMEM, while a caller-supplied workspace still runs.
After each injected failure the same context solves normally again.
"""
import numpy as np
import pytest
import torch

import ct_inputs as ci

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_07408_gb300 import ct as _ct
    yield _ct
    _ct.fault_set(None)


@pytest.fixture(scope="module")
def scan(ct):
    spec = ci.CONE_ANISO
    x = ci.phantom(spec)[0]
    g = ct.Geometry.from_spec(spec)
    b = ct.project_A(g, torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    return spec, g, b


def test_nan_in_host_data_stops_before_the_first_iteration(ct, scan):
    spec, g, b = scan
    bh = b.cpu().clone().pin_memory()
    bh.view(-1)[12345 % spec.m] = float("nan")
    xh = torch.zeros(spec.vol_shape).pin_memory()
    with pytest.raises(ct.CTError) as ei:
        ct.ct_bagmres_solve_host(g, bh, 6, xh, ct.make_opts(b_kind="fbp"))
    assert ei.value.status == ct.CT_ENONFINITE
    r = ei.value.result
    assert r.iters == 0 and np.isnan(r.resid[0]) and np.all(r.resid[1:] == -1.0)
    # the context is intact: the clean data solves
    res = ct.ct_bagmres_solve_host(g, b.cpu().pin_memory(), 6, xh, ct.make_opts(b_kind="fbp"))
    assert res.iters == 6 and np.all(np.isfinite(res.resid))


SOLVERS = {
    "ba": lambda ct, g, b, x, k: ct.ct_bagmres_solve(g, b, k, x, ct.make_opts(b_kind="un")),
    "ab": lambda ct, g, b, x, k: ct.ct_abgmres_solve(g, b, k, x, ct.make_opts(b_kind="fbp")),
    "cgls": lambda ct, g, b, x, k: ct.ct_cgls_solve(g, b, k, x, ct.make_opts(b_kind="un")),
}


@pytest.mark.parametrize("solver", sorted(SOLVERS))
def test_nan_injected_at_iteration_stops_the_solve(ct, scan, solver):
    spec, g, b = scan
    k, n_bad = 8, 4
    run = SOLVERS[solver]
    x = torch.empty(spec.vol_shape, device="cuda")
    ct.fault_set(None)
    clean = run(ct, g, b, x, k)
    ct.fault_set("nan_at_iter:%d" % n_bad)
    assert ct.fault_get() == "nan_at_iter:%d" % n_bad
    try:
        with pytest.raises(ct.CTError) as ei:
            run(ct, g, b, x, k)
    finally:
        ct.fault_set(None)
    assert ei.value.status == ct.CT_ENONFINITE
    r = ei.value.result
    assert r.iters == n_bad - 1
    np.testing.assert_array_equal(r.resid[:n_bad], clean.resid[:n_bad])
    assert np.all(r.resid[n_bad:] == -1.0)
    again = run(ct, g, b, x, k)
    np.testing.assert_array_equal(again.resid, clean.resid)


def test_nan_injected_in_the_adjoint_gmres(ct, scan):
    spec, g, _ = scan
    gx = torch.from_numpy(ci.random_vector(spec.n, 3).astype(np.float32).reshape(spec.vol_shape)).cuda()
    gb = torch.empty(spec.sino_shape, device="cuda")
    ct.fault_set("nan_at_iter:2")
    try:
        with pytest.raises(ct.CTError) as ei:
            ct.ct_bagmres_vjp(g, gx, 5, gb, ct.make_opts(b_kind="un"))
    finally:
        ct.fault_set(None)
    assert ei.value.status == ct.CT_ENONFINITE and ei.value.result.iters == 1
    assert np.all(ei.value.result.resid[2:] == -1.0)


def test_injected_allocation_failure(ct, scan):
    spec, g, b = scan
    x = torch.empty(spec.vol_shape, device="cuda")
    ct.fault_set("oom")
    try:
        with pytest.raises(ct.CTError) as ei:
            ct.ct_bagmres_solve(g, b, 3, x, ct.make_opts(), workspace=None)
        assert ei.value.status == ct.CT_ENOMEM and "CT_FAULT" in str(ei.value)
        with pytest.raises(ct.CTError) as ei:
            ct.ct_project_A(g, x, torch.empty(spec.sino_shape, device="cuda"))
        assert ei.value.status == ct.CT_ENOMEM
        # a caller workspace does not go through the allocator
        res = ct.ct_bagmres_solve(g, b, 3, x, ct.make_opts(), workspace="torch")
        assert res.iters == 3
    finally:
        ct.fault_set(None)
    res = ct.ct_bagmres_solve(g, b, 3, x, ct.make_opts(), workspace=None)
    assert res.iters == 3

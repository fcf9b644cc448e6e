"""Concurrent use of the library: solves and operator calls issued from
several host threads, each on its own CUDA stream, against one shared
geometry and against separate ones.  The library keeps no mutable state
across calls besides the per-call workspaces (stream-ordered allocations or
caller workspaces), the profiler (behind a mutex) and the thread-local error
message, so every concurrent result must equal, bit for bit, the same call
made alone.
"""
import threading

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
    return _ct


def data(ct, g, spec, seed):
    x = torch.from_numpy(ci.phantom(spec, seed=seed)[0]).cuda()
    b = ct.project_A(g, x)
    torch.cuda.synchronize()
    return b


def run_threads(fns):
    errors = []

    def wrap(fn):
        try:
            fn()
        except Exception as e:   # reported below, with the thread's failure
            errors.append(e)

    threads = [threading.Thread(target=wrap, args=(fn,)) for fn in fns]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not any(t.is_alive() for t in threads), "a solve did not finish"
    assert not errors, errors


def test_concurrent_solves_equal_sequential_ones(ct):
    specs = [ci.CONE_SMALL, ci.CONE_ANISO, ci.CONE_SMALL, ci.PAR2D_ANISO]
    geoms = {s.name: ct.Geometry.from_spec(s) for s in specs}
    shared = geoms[ci.CONE_SMALL.name]   # two of the threads share this geometry
    jobs = []
    for i, spec in enumerate(specs):
        g = shared if spec is ci.CONE_SMALL else geoms[spec.name]
        b = data(ct, g, spec, seed=i)
        kind = ("un", "fbp")[i % 2]
        jobs.append((spec, g, b, kind))
    # alone
    ref = []
    for spec, g, b, kind in jobs:
        x = torch.empty(spec.vol_shape, device="cuda")
        r = ct.ct_bagmres_solve(g, b, 10, x, ct.make_opts(b_kind=kind))
        ref.append((x.clone(), r.resid.copy()))
    # together, each thread on its own stream, three rounds
    out = [None] * len(jobs)

    def solve(i):
        spec, g, b, kind = jobs[i]
        st = torch.cuda.Stream()
        for _ in range(3):
            x = torch.empty(spec.vol_shape, device="cuda")
            r = ct.ct_bagmres_solve(g, b, 10, x, ct.make_opts(b_kind=kind), stream=st)
            st.synchronize()
            out[i] = (x, r.resid.copy())
    run_threads([lambda i=i: solve(i) for i in range(len(jobs))])
    for (x, r), (x0, r0) in zip(out, ref):
        assert torch.equal(x, x0)
        assert np.array_equal(r, r0)


def test_concurrent_operator_calls_equal_sequential_ones(ct):
    spec = ci.CONE_ANISO
    g = ct.Geometry.from_spec(spec)
    xs = [torch.from_numpy(ci.random_vector(spec.n, seed=20 + i, positive=True).astype(np.float32)
                           .reshape(spec.vol_shape)).cuda() for i in range(4)]
    ref = []
    for x in xs:
        y = ct.project_A(g, x)
        ref.append((y.clone(), ct.backproject_B(g, y, "fbp").clone()))
    torch.cuda.synchronize()
    out = [None] * len(xs)

    def work(i):
        st = torch.cuda.Stream()
        y = torch.empty(spec.sino_shape, device="cuda")
        v = torch.empty(spec.vol_shape, device="cuda")
        for _ in range(5):
            ct.ct_project_A(g, xs[i], y, stream=st)
            ct.ct_backproject_B(g, y, v, "fbp", stream=st)
        st.synchronize()
        out[i] = (y, v)
    run_threads([lambda i=i: work(i) for i in range(len(xs))])
    for (y, v), (y0, v0) in zip(out, ref):
        assert torch.equal(y, y0) and torch.equal(v, v0)


def test_concurrent_operators_on_geometries_of_different_view_counts(ct):
    """The back-projector's shared memory grows with the view count, and a
    kernel's shared-memory limit is process-wide: threads running the same
    kernels on geometries with 60, 45 and 36 views (each on its own stream)
    must all launch, and give what the same calls give alone."""
    specs = [ci.CONE_SMALL, ci.CONE_ANISO, ci.CONE_THIN, ci.CONE_SMALL, ci.CONE_ANISO, ci.CONE_THIN]
    geoms = [ct.Geometry.from_spec(s) for s in specs]
    ys = [data(ct, g, s, seed=30 + i) for i, (g, s) in enumerate(zip(geoms, specs))]
    ref = [(ct.backproject_B(g, y, "fbp").clone(), ct.adjoint_Bt(g, ct.backproject_B(g, y), "un").clone())
           for g, y in zip(geoms, ys)]
    torch.cuda.synchronize()
    out = [None] * len(specs)

    def work(i):
        g, y, spec = geoms[i], ys[i], specs[i]
        st = torch.cuda.Stream()
        v = torch.empty(spec.vol_shape, device="cuda")
        w = torch.empty(spec.sino_shape, device="cuda")
        for _ in range(20):
            ct.ct_backproject_B(g, y, v, "fbp", stream=st)
        u = torch.empty(spec.vol_shape, device="cuda")
        ct.ct_backproject_B(g, y, u, "un", stream=st)
        ct.ct_adjoint_Bt(g, u, w, "un", stream=st)
        st.synchronize()
        out[i] = (v, w)
    run_threads([lambda i=i: work(i) for i in range(len(specs))])
    for (v, w), (v0, w0) in zip(out, ref):
        assert torch.equal(v, v0)
        # B^T accumulates with FP32 atomics: equal up to summation order
        assert float((w - w0).norm() / w0.norm()) <= 1e-6

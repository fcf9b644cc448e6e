"""The persistent BA-GMRES state (ct_bagmres_state_*, ct_gmres_state_*): a
solve that can be extended, saved and restored, with its Krylov basis in
device memory or in page-locked host memory (Sec. II keeps the growing
basis outside the solver's working memory, on disk).

The state runs the same kernels in the same order as ct_bagmres_solve, so
the checks are bitwise:
  * k iterations split over several extend calls give the image and the
    residual history of one k-iteration solve;
  * extending to a k below the iterations done forms that earlier iterate,
    equal to a solve with that k;
  * a state saved after some iterations, destroyed and loaded again (with a
    larger capacity, with its basis on the host or the device) continues to
    the same result as one uninterrupted solve;
  * a host-resident basis gives the device basis's result.
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
    return _ct


def scan(ct, spec, storage="f32"):
    g = ct.Geometry.from_spec(spec, vol_dtype=storage, sino_dtype=storage)
    x = torch.from_numpy(ci.phantom(spec)[0]).cuda()
    b = ct.project_A(g, x)
    b = b + 0.01 * float(b.max()) * torch.from_numpy(
        ci.gaussian_noise(spec.sino_shape, 1.0, seed=4).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    return g, b


def one_call(ct, g, spec, b, k, b_kind):
    x = torch.empty(spec.vol_shape, device="cuda")
    res = ct.ct_bagmres_solve(g, b, k, x, ct.make_opts(b_kind=b_kind))
    return x, res


CASES = [(ci.CONE_ANISO, "f32", "fbp"), (ci.CONE_ANISO, "f32", "un"), (ci.CONE_SMALL, "bf16", "un"),
         (ci.PAR2D_ANISO, "f32", "fbp")]


@pytest.mark.parametrize("spec,storage,b_kind", CASES, ids=lambda v: getattr(v, "name", str(v)))
@pytest.mark.parametrize("basis", ["device", "host"])
def test_extend_in_steps_equals_one_solve(ct, spec, storage, b_kind, basis):
    g, b = scan(ct, spec, storage)
    x12, r12 = one_call(ct, g, spec, b, 12, b_kind)
    x5, r5 = one_call(ct, g, spec, b, 5, b_kind)
    st = ct.GmresState(g, 12, basis, ct.make_opts(b_kind=b_kind))
    st.start(b)
    x = torch.empty(spec.vol_shape, device="cuda")
    ra = st.extend(5, x)
    assert st.iters == 5 and ra.iters == 5
    assert torch.equal(x, x5) and np.array_equal(ra.resid, r5.resid)
    rb = st.extend(12, x)
    assert st.iters == 12 and rb.iters == 12
    assert torch.equal(x, x12) and np.array_equal(rb.resid, r12.resid)
    # an earlier iterate from the grown basis
    rc = st.extend(5, x)
    assert st.iters == 12 and rc.iters == 5
    assert torch.equal(x, x5) and np.array_equal(rc.resid, r5.resid)
    st.close()


@pytest.mark.parametrize("basis_before,basis_after", [("device", "device"), ("device", "host"), ("host", "device")])
def test_save_and_load_resume_the_solve(ct, tmp_path, basis_before, basis_after):
    spec, b_kind = ci.CONE_ANISO, "fbp"
    g, b = scan(ct, spec)
    x14, r14 = one_call(ct, g, spec, b, 14, b_kind)
    st = ct.GmresState(g, 8, basis_before, ct.make_opts(b_kind=b_kind))
    st.start(b)
    x = torch.empty(spec.vol_shape, device="cuda")
    st.extend(6, x)
    path = tmp_path / "state.ctg"
    st.save(path)
    st.close()
    st2 = ct.GmresState.load(g, path, 14, basis_after)
    assert st2.iters == 6
    r = st2.extend(14, x)
    assert torch.equal(x, x14) and np.array_equal(r.resid, r14.resid)
    st2.close()


def test_load_rejects_another_geometry_and_a_small_capacity(ct, tmp_path):
    spec = ci.CONE_ANISO
    g, b = scan(ct, spec)
    st = ct.GmresState(g, 6, "device", ct.make_opts(b_kind="un"))
    st.start(b)
    x = torch.empty(spec.vol_shape, device="cuda")
    st.extend(6, x)
    path = tmp_path / "state.ctg"
    st.save(path)
    other = ct.Geometry.from_spec(ci.scaled(spec, n_views=spec.n_views + 1))
    with pytest.raises(ct.CTError) as ei:
        ct.GmresState.load(other, path, 10)
    assert ei.value.status == ct.CT_EINVAL and "geometry" in str(ei.value)
    with pytest.raises(ct.CTError) as ei:
        ct.GmresState.load(g, path, 5)
    assert ei.value.status == ct.CT_EINVAL
    with pytest.raises(ct.CTError):
        st.extend(7, x)            # beyond kmax
    bad = tmp_path / "junk.ctg"
    bad.write_bytes(b"not a state")
    with pytest.raises(ct.CTError):
        ct.GmresState.load(g, bad, 10)
    st.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_host_basis_with_second_sweep_equals_one_solve(ct, storage):
    """The host basis comes back to the device through a ring of buffers for
    every MGS sweep, the optional second sweep included, and for the final
    x = V y: still the one-call solve's bits."""
    spec = ci.CONE_ANISO
    g, b = scan(ct, spec, storage)
    opts = ct.make_opts(b_kind="un", reorth=1)
    x1 = torch.empty(spec.vol_shape, device="cuda")
    r1 = ct.ct_bagmres_solve(g, b, 9, x1, opts)
    st = ct.GmresState(g, 9, "host", ct.make_opts(b_kind="un", reorth=1))
    st.start(b)
    x = torch.empty(spec.vol_shape, device="cuda")
    st.extend(4, x)
    r = st.extend(9, x)
    assert torch.equal(x, x1) and np.array_equal(r.resid, r1.resid)
    st.close()

"""The projector entry point that allocates nothing: ct_project_A_noalloc.

It exists for callers that cannot allocate device memory while they run (a
TensorRT plugin inside enqueue(), a framework that reserved all device
memory for its own pool, a real-time loop that must not risk allocation
latency or failure).  It takes its scratch from a fixed array that the
library keeps in device memory.  These checks call it through the C-ABI and
compare it with the allocating ct_project_A, within the operator tolerance
of the other GPU tests, on two calls in a row with different inputs (after
a call on another grid has left non-zero values in the scratch), and check
that a volume too large for the fixed scratch is refused.  The file
is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import ct_inputs as ci

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


@pytest.fixture(scope="module")
def ct():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_07408_gb300 import ct as _ct
    return _ct


def _call_noalloc(ct, g, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ct.lib().ct_project_A_noalloc(g.handle, ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(y.data_ptr()), stream)


def _check_against_allocating(ct, g, spec, x_host):
    x = torch.from_numpy(np.ascontiguousarray(x_host, dtype=np.float32).reshape(spec.vol_shape)).cuda()
    ref = torch.empty(spec.sino_shape, device="cuda")
    ct.ct_project_A(g, x, ref)
    out = torch.full(spec.sino_shape, float("nan"), device="cuda")
    assert _call_noalloc(ct, g, x, out) == ct.CT_OK, ct.lib().ct_last_error()
    torch.cuda.synchronize()
    err = float((out.double() - ref.double()).norm() / ref.double().norm())
    assert err <= OP_TOL, err
    assert not torch.isnan(out).any()


def test_noalloc_projector_matches_allocating_projector(ct):
    # First a call on a larger grid of another shape with a positive volume:
    # it leaves non-zero values across the part of the scratch that the
    # 128^3 copies use, where their zero borders fall on other positions, so
    # a border that a later call failed to rewrite would show.
    pre = ci._cone("noalloc_prefill", 0, 0.8, 40, 220, 170, 1.2, nxyz=(150, 140, 150))
    _check_against_allocating(ct, ct.Geometry.from_spec(pre), pre,
                              ci.random_vector(pre.n, seed=9, positive=True) + 0.5)
    spec = ci.CONE_128
    g = ct.Geometry.from_spec(spec)
    inputs = [ci.phantom(spec)[0], ci.random_vector(spec.n, seed=5, positive=True).astype(np.float32)]
    for x_host in inputs:   # two calls in a row; the second sees the first call's scratch
        _check_against_allocating(ct, g, spec, x_host)


def test_noalloc_projector_refuses_a_volume_beyond_its_scratch(ct):
    spec = ci.CONE_256
    g = ct.Geometry.from_spec(spec)
    x = torch.zeros(spec.vol_shape, device="cuda")
    y = torch.zeros(spec.sino_shape, device="cuda")
    assert _call_noalloc(ct, g, x, y) == ct.CT_EINVAL
    assert b"scratch" in ct.lib().ct_last_error()

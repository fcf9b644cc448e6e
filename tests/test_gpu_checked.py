"""The index-checked build (libct_checked.so) on the GPU.

Every operator and solver on the small and degenerate scans (FP32 and BF16
storage, both projectors) must leave no failed check: the row margin of the
back-projector, the projector's z border and row window, and the
line-intersection walk's voxel offsets hold on every sample.  Then each check is shown to fire when
its precondition is removed on the host, in the checked build only:

* CT_DEBUG_PADV=2 shrinks the back-projector's row margin on cone_small
  (the host sizes it at 22 rows there), so voxels near the top and bottom
  slices project outside their view's padded rows: site 4 (B row);
* CT_DEBUG_A_ZSAFE=1 tells the projector that no z clamp is needed on a
  scan whose detector rows reach far beyond its 8 slices: site 1 (A z).

A failed check redirects the access into range before it is made, so these
runs read nothing outside their buffers.  Each runs in a child process
(tests/checked_run.py) so that only the checked library is loaded there.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = os.path.join(ROOT, "tests", "checked_run.py")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def run(mode, **env):
    e = dict(os.environ)
    e.pop("CT_DEBUG_PADV", None)
    e.pop("CT_DEBUG_A_ZSAFE", None)
    e.update(env)
    e["CT_LIB"] = "checked"
    r = subprocess.run([sys.executable, SCRIPT, mode], capture_output=True, text=True, env=e, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_check_fails_on_any_operator_or_solver():
    res = run("all")
    assert len(res) == 31
    failed = {case: [(name, rec) for name, rec in calls if rec is not None] for case, calls in res.items()}
    failed = {k: v for k, v in failed.items() if v}
    assert not failed, failed


def test_no_check_fails_on_random_scans():
    res = run("random")
    failed = {case: [(name, rec) for name, rec in calls if rec is not None] for case, calls in res.items()}
    failed = {k: v for k, v in failed.items() if v}
    assert len(res) > 40 and not failed, failed


def test_row_check_fires_when_the_margin_is_too_small():
    res = run("margin", CT_DEBUG_PADV="2")
    assert res["A"] is None
    site, view, row = res["B_un"]
    assert site == 4
    assert 0 <= view < 60
    # the offending quad row lies outside the view's 44 + 2 * 2 padded rows
    assert row < 0 or row >= 48


def test_z_check_fires_when_the_projector_skips_its_clamp():
    res = run("zsafe", CT_DEBUG_A_ZSAFE="1")
    site, view, z = res["A"]
    assert site == 1
    assert 0 <= view < 30
    # outside [-PAD_A, nz + PAD_A - 2] = [-2, 8]
    assert z < -2 or z > 8

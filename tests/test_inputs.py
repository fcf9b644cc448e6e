"""The seeded input generators: random scans are valid for the library
(source outside the grid's circle, detector behind the source) and
reproducible."""
import math

import ct_inputs as ci


def test_random_scans_are_valid_and_reproducible():
    kinds = set()
    for seed in range(24):
        g = ci.random_geometry(seed)
        assert g == ci.random_geometry(seed)
        kinds.add(g.kind)
        assert min(g.nx, g.ny, g.nz, g.n_views, g.nu, g.nv) >= 1
        if g.kind == ci.CONE_3D:
            r = math.hypot(0.5 * g.nx * g.vox, 0.5 * g.ny * g.vox)
            assert g.sod > r and g.sdd > g.sod
        else:
            assert g.nz == 1 and g.nv == 1
    assert kinds == {ci.CONE_3D, ci.PARALLEL_2D}

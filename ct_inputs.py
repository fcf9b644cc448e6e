"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds the workload descriptions (scan geometries) and the seeded
random generators (phantoms, noise, random vectors).  It contains none of the
reconstruction method's arithmetic: no projector, no back-projector, no filter
and no Krylov step.  Both sides of every parity check draw their inputs here.

The paper's data (a veterinary cone-beam scan of a QA phantom, 180 of 720 views
on a 1088x896 detector, Sec. III) is not available; these phantoms and
geometries stand in for it.  The 3D scans follow the paper's circular
cone-beam set-up (Sec. III): one full rotation, flat detector.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, replace

import numpy as np

PARALLEL_2D = 0
CONE_3D = 1


@dataclass(frozen=True)
class Geometry:
    """Scan and grid description (all lengths in mm, angles in radians).

    Volume: nx*ny*nz voxels of edge ``vox``, centred on the rotation axis,
    stored vol[z][y][x] (x fastest).  Views: theta_s = ang0 + s*span/n_views.
    Detector: nu*nv pixels of size du*dv centred on the central ray, stored
    sino[view][v][u] (u fastest).  Cone beam: source at distance ``sod`` from
    the axis, detector at distance ``sdd`` from the source.  2D parallel beam:
    nz = nv = 1 and sod/sdd unused.
    """

    name: str
    kind: int
    nx: int
    ny: int
    nz: int
    vox: float
    n_views: int
    ang0: float
    span: float
    nu: int
    nv: int
    du: float
    dv: float
    sod: float = 0.0
    sdd: float = 0.0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def m(self) -> int:
        return self.n_views * self.nv * self.nu

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.n_views, self.nv, self.nu)

    def as_dict(self):
        return asdict(self)

    def joseph_samples(self) -> int:
        """Nominal Joseph sample count of one A: rays x dominant-axis planes.

        Every ray walks max(nx, ny) planes when nx == ny; for non-square grids
        the count depends on each ray's dominant axis, so the nominal figure
        uses the larger in-plane dimension.
        """
        return self.m * max(self.nx, self.ny)

    def voxel_view_samples(self) -> int:
        """Voxel-view pairs of one voxel-driven B: voxels x views."""
        return self.n * self.n_views


def _cone(name, nvox, vox, n_views, nu, nv, det, sod=500.0, sdd=1000.0, ang0=0.0,
          span=2 * math.pi, nxyz=None, dv=None):
    nx, ny, nz = nxyz if nxyz else (nvox, nvox, nvox)
    return Geometry(name=name, kind=CONE_3D, nx=nx, ny=ny, nz=nz, vox=vox,
                    n_views=n_views, ang0=ang0, span=span, nu=nu, nv=nv,
                    du=det, dv=det if dv is None else dv, sod=sod, sdd=sdd)


# --- the workloads -----------------------------------------------------------
# 2D parallel beam, 64x64 pixels of 1, 90 views over 180 deg, 95 bins of 1.
PAR2D_64 = Geometry(name="par2d_64", kind=PARALLEL_2D, nx=64, ny=64, nz=1, vox=1.0,
                    n_views=90, ang0=0.0, span=math.pi, nu=95, nv=1, du=1.0, dv=1.0)
# 3D circular cone beam, 128^3 voxels of 1 mm, 128 views over 360 deg,
# 192x128 detector of 1.5 mm, SOD 500 mm, SDD 1000 mm.
CONE_128 = _cone("cone_128", 128, 1.0, 128, 192, 128, 1.5)
# The same field of view at 256^3 (0.5 mm), 360 views, 384x256 detector (0.75 mm).
CONE_256 = _cone("cone_256", 256, 0.5, 360, 384, 256, 0.75)
# The same field of view at 512^3 (0.25 mm), 720 views, 768x512 detector (0.375 mm).
CONE_512 = _cone("cone_512", 512, 0.25, 720, 768, 512, 0.375)
# 64^3 cut-down of the 512^3 scan: 2 mm voxels, 96x64 detector of 3 mm, 90 views.
CONE_512_CUT64 = _cone("cone_512_cut64", 64, 2.0, 90, 96, 64, 3.0)
# 32^3 gradient-check scan: 4 mm voxels, 48x32 detector of 6 mm, 128 views.
CONE_GRAD32 = _cone("cone_grad32", 32, 4.0, 128, 48, 32, 6.0)

# Small parity cases that the oracle finishes in seconds.  Sizes are chosen
# off the kernels' tile sizes (ragged tails) and non-cubic grids catch
# transposed indices.
CONE_SMALL = _cone("cone_small", 44, 128.0 / 44, 60, 66, 44, 288.0 / 66)
CONE_ANISO = _cone("cone_aniso", 0, 3.0, 45, 70, 30, 4.0, nxyz=(40, 36, 28),
                   ang0=0.3, dv=4.5)
# a slab thinner than the back-projector's z run (5 slices) on a detector
# whose row count (7) is not a multiple of the projector's rays per thread
CONE_THIN = _cone("cone_thin", 0, 2.5, 36, 50, 7, 3.5, nxyz=(30, 26, 5), ang0=0.2)
PAR2D_ANISO = Geometry(name="par2d_aniso", kind=PARALLEL_2D, nx=37, ny=29, nz=1,
                       vox=1.3, n_views=41, ang0=0.1, span=math.pi, nu=53, nv=1,
                       du=1.1, dv=1.0)
# 40 slices: the last 16-slice run of the bf16 back-projector passes nz by 8
# slices (the row margin must cover them), while 8-slice runs end at nz
CONE_Z40 = _cone("cone_z40", 40, 3.0, 48, 66, 44, 4.5, ang0=0.15)

# Degenerate scans: one voxel; one view; a one-row cone-beam detector; a
# one-voxel-wide column of slices; a 2D scan with three detector bins.
CONE_VOXEL1 = _cone("cone_voxel1", 1, 10.0, 3, 5, 5, 8.0, ang0=0.2)
CONE_1VIEW = _cone("cone_1view", 0, 3.0, 1, 20, 14, 5.0, nxyz=(12, 10, 9), ang0=0.4)
CONE_1ROW = _cone("cone_1row", 0, 2.0, 24, 30, 1, 2.5, nxyz=(16, 16, 6), dv=4.0)
CONE_COLUMN = _cone("cone_column", 0, 2.0, 8, 6, 30, 3.0, nxyz=(1, 1, 24), ang0=0.1)
PAR2D_3BIN = Geometry(name="par2d_3bin", kind=PARALLEL_2D, nx=9, ny=7, nz=1, vox=1.0,
                      n_views=5, ang0=0.0, span=math.pi, nu=3, nv=1, du=4.0, dv=1.0)
DEGENERATE = [CONE_VOXEL1, CONE_1VIEW, CONE_1ROW, CONE_COLUMN, PAR2D_3BIN]

def random_geometry(seed: int) -> Geometry:
    """A seeded random small scan within the library's limits, for parity
    sweeps over shapes the named scans do not cover: grids of 1..40 voxels
    per axis, 1..70 views over a span of 0.3..2 pi from any start angle,
    source distances of 100..800 mm with magnification 1.1..3, detectors
    covering 0.5..1.6 of the volume's shadow with pixel aspect 0.6..1.6;
    every fifth one is a 2D parallel-beam scan."""
    rng = np.random.default_rng(1000 + seed)
    nx, ny = (int(v) for v in rng.integers(1, 41, size=2))
    vox = float(rng.uniform(0.5, 4.0))
    n_views = int(rng.integers(1, 71))
    span = float(2 * math.pi if rng.random() < 0.5 else rng.uniform(0.3, 2 * math.pi))
    ang0 = float(rng.uniform(0.0, 2 * math.pi))
    half = 0.5 * vox * math.hypot(nx, ny)
    if seed % 5 == 4:
        nu = int(rng.integers(3, 97))
        du = float(2 * half * rng.uniform(0.5, 1.6) / nu)
        return Geometry(name="random%d" % seed, kind=PARALLEL_2D, nx=nx, ny=ny, nz=1, vox=vox,
                        n_views=n_views, ang0=ang0, span=span, nu=nu, nv=1, du=du, dv=1.0)
    nz = int(rng.integers(1, 41))
    sod = float(max(rng.uniform(100.0, 800.0), 1.5 * half + 10.0))
    sdd = float(sod * rng.uniform(1.1, 3.0))
    mag = sdd / sod
    nu = int(rng.integers(3, 97))
    nv = int(rng.integers(1, 65))
    du = float(2 * half * mag * rng.uniform(0.5, 1.6) / nu)
    dv = float(du * rng.uniform(0.6, 1.6))
    return Geometry(name="random%d" % seed, kind=CONE_3D, nx=nx, ny=ny, nz=nz, vox=vox, n_views=n_views,
                    ang0=ang0, span=span, nu=nu, nv=nv, du=du, dv=dv, sod=sod, sdd=sdd)


WORKLOADS = {g.name: g for g in (PAR2D_64, CONE_128, CONE_256, CONE_512, CONE_512_CUT64,
                                 CONE_GRAD32, CONE_SMALL, CONE_ANISO, CONE_THIN, PAR2D_ANISO,
                                 CONE_Z40, *DEGENERATE)}


def scaled(g: Geometry, **kw) -> Geometry:
    """A copy of ``g`` with some fields replaced."""
    return replace(g, **kw)


# --- phantoms ----------------------------------------------------------------
@dataclass
class Ellipsoid:
    centre: np.ndarray    # (3,) mm
    semi: np.ndarray      # (3,) semi-axes, mm
    rot: np.ndarray       # (3,3) columns = principal axes in world coordinates
    density: float        # 1/mm (attenuation), added where ellipsoids overlap


def _random_rotation(rng) -> np.ndarray:
    """Uniform rotation on SO(3) from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def random_ellipsoids(n_ell=12, seed=0, z_half=40.0, r_max=55.0, semi_range=(5.0, 30.0),
                      dens_range=(0.0, 0.02), scale=1.0):
    """Seeded ellipsoids confined to the cylinder |z| <= z_half, radius <= r_max.

    Semi-axes are uniform in ``semi_range``, orientation uniform on SO(3),
    density uniform in ``dens_range``; each ellipsoid's bounding box lies
    inside the cylinder.  ``scale`` shrinks all lengths (for small grids).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_ell):
        semi = rng.uniform(*semi_range, size=3) * scale
        rot = _random_rotation(rng)
        # half-extent of the ellipsoid along each world axis
        ext = np.sqrt(((rot * semi[None, :]) ** 2).sum(axis=1))
        ez = ext[2]
        er = math.hypot(ext[0], ext[1])
        zc = rng.uniform(-(z_half * scale - ez), z_half * scale - ez)
        rr = (r_max * scale - er) * math.sqrt(rng.uniform(0, 1))
        ph = rng.uniform(0, 2 * math.pi)
        centre = np.array([rr * math.cos(ph), rr * math.sin(ph), zc])
        dens = float(rng.uniform(*dens_range))
        out.append(Ellipsoid(centre=centre, semi=semi, rot=rot, density=dens))
    return out


def random_ellipses_2d(n_ell=10, seed=0, radius=28.0):
    """Shepp-Logan-style 2D phantom: an outer skull ellipse (density 1), a
    slightly smaller brain ellipse (density -0.8 relative, giving 0.2 inside),
    and eight seeded interior ellipses with densities in [0, 0.8] relative;
    total densities stay in [0, 1].  Returned as 3D ellipsoids with z-axis
    semi-axis infinity-like (the 2D phantom is a z-invariant cylinder)."""
    rng = np.random.default_rng(seed)
    big = 1e6
    out = [Ellipsoid(np.zeros(3), np.array([0.92 * radius, 0.72 * radius, big]), np.eye(3), 1.0),
           Ellipsoid(np.zeros(3), np.array([0.86 * radius, 0.66 * radius, big]), np.eye(3), -0.8)]
    for _ in range(n_ell - 2):
        a, b = rng.uniform(0.06, 0.3, size=2) * radius
        ang = rng.uniform(0, math.pi)
        c, s = math.cos(ang), math.sin(ang)
        rot = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
        lim = 0.55 * radius - max(a, b)
        rr = max(lim, 0.0) * math.sqrt(rng.uniform(0, 1))
        ph = rng.uniform(0, 2 * math.pi)
        cen = np.array([rr * 1.2 * math.cos(ph), rr * 0.9 * math.sin(ph), 0.0])
        out.append(Ellipsoid(cen, np.array([a, b, big]), rot, float(rng.uniform(0.0, 0.8))))
    return out


def voxel_centres(g: Geometry):
    """Voxel-centre coordinates (mm) along x, y, z: (i - (N-1)/2) * vox."""
    xs = (np.arange(g.nx) - (g.nx - 1) / 2.0) * g.vox
    ys = (np.arange(g.ny) - (g.ny - 1) / 2.0) * g.vox
    zs = (np.arange(g.nz) - (g.nz - 1) / 2.0) * g.vox
    return xs, ys, zs


def voxelize(g: Geometry, ells, dtype=np.float32, supersample=1):
    """Sum of ellipsoid indicator * density sampled at voxel centres (or the
    mean over supersample^3 points per voxel), shape (nz, ny, nx)."""
    xs, ys, zs = voxel_centres(g)
    vol = np.zeros(g.vol_shape, dtype=np.float64)
    offs = (np.arange(supersample) + 0.5) / supersample - 0.5
    sub_z = offs if g.nz > 1 else np.zeros(1)
    for dz in sub_z:
        for dy in offs:
            for dx in offs:
                X = (xs + dx * g.vox)[None, None, :]
                Y = (ys + dy * g.vox)[None, :, None]
                for k0 in range(0, g.nz, 64):
                    Z = (zs[k0:k0 + 64] + dz * g.vox)[:, None, None]
                    acc = vol[k0:k0 + 64]
                    for e in ells:
                        # coordinates in the ellipsoid frame: rot^T (r - c)
                        px, py, pz = X - e.centre[0], Y - e.centre[1], Z - e.centre[2]
                        q = 0.0
                        for ax in range(3):
                            comp = (e.rot[0, ax] * px + e.rot[1, ax] * py + e.rot[2, ax] * pz)
                            q = q + (comp / e.semi[ax]) ** 2
                        acc += np.where(q <= 1.0, e.density, 0.0) / (len(offs) ** 2 * len(sub_z))
    return vol.astype(dtype)


def phantom(g: Geometry, seed=0, dtype=np.float32):
    """The workload's phantom: 10 seeded ellipses (2D) or 12 seeded
    ellipsoids in the axially confined cylinder (3D), scaled to the grid's
    field of view (the 128 mm field at 1 mm voxels is the unit)."""
    if g.kind == PARALLEL_2D:
        ells = random_ellipses_2d(10, seed=seed, radius=0.5 * min(g.nx, g.ny) * g.vox)
    else:
        fov = min(g.nx, g.ny) * g.vox
        z_half = min(40.0, 0.45 * g.nz * g.vox * 128.0 / fov)
        # slabs thinner than the largest ellipsoid get proportionally smaller ones
        semi = (5.0, 30.0) if z_half > 34.0 else (0.15 * z_half, 0.85 * z_half)
        ells = random_ellipsoids(12, seed=seed, scale=fov / 128.0, z_half=z_half, semi_range=semi)
    return voxelize(g, ells, dtype=dtype), ells


# --- noise and random vectors ---------------------------------------------------
def gaussian_noise(shape, sigma, seed=1, dtype=np.float64):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) * sigma).astype(dtype)


def poisson_log_data(line_integrals, i0=1e5, seed=1, dtype=np.float32):
    """Photon counts ~ Poisson(i0 * exp(-p)), clamped to >= 1, then
    b = -log(counts / i0): the negative-log preprocessing of Sec. I."""
    rng = np.random.default_rng(seed)
    p = np.asarray(line_integrals, dtype=np.float64)
    counts = rng.poisson(i0 * np.exp(-p))
    counts = np.maximum(counts, 1)
    return (-np.log(counts / i0)).astype(dtype)


def random_vector(size, seed, dtype=np.float64, positive=False):
    rng = np.random.default_rng(seed)
    v = rng.uniform(0.0, 1.0, size) if positive else rng.standard_normal(size)
    return v.astype(dtype)


def smooth_volume(g: Geometry, seed=3, dtype=np.float64):
    """A smooth positive volume (sum of a few wide Gaussians), for scale checks."""
    rng = np.random.default_rng(seed)
    xs, ys, zs = voxel_centres(g)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    fov = min(g.nx, g.ny) * g.vox
    vol = np.zeros(g.vol_shape)
    for _ in range(4):
        c = rng.uniform(-0.2, 0.2, 3) * fov
        if g.nz == 1:
            c[2] = 0.0
        s = rng.uniform(0.15, 0.3) * fov
        vol += np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * s * s))
    return vol.astype(dtype)


def sample_indices(total, count, seed=2):
    """Seeded sorted distinct indices in [0, total)."""
    rng = np.random.default_rng(seed)
    count = min(count, total)
    return np.sort(rng.choice(total, size=count, replace=False)).astype(np.int64)

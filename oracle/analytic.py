"""Closed-form line integrals for pinning the projector (test infrastructure).

The line integral of an ellipsoid of constant density along a straight line
is the density times the chord length, which has a closed form: with the
line S + t d mapped into the ellipsoid's unit-sphere frame (p0 + t q), the
chord spans the roots of |p0 + t q|^2 = 1.  A Joseph projector applied to a
voxelised phantom converges to these values as the grid is refined, so they
pin A (Sec. I Eq. 1: A models line integration) independently of any
discretisation.
"""
from __future__ import annotations

import numpy as np


def ray_geometry(g, rays=None):
    """Source points S (R,3) and unit directions (R,3) of the listed rays,
    built from the scan description by plain vector geometry."""
    if rays is None:
        rays = np.arange(g.m)
    rays = np.asarray(rays, dtype=np.int64)
    s = rays // (g.nu * g.nv)
    iv = (rays % (g.nu * g.nv)) // g.nu
    iu = rays % g.nu
    th = g.ang0 + s * g.span / g.n_views
    c, sn = np.cos(th), np.sin(th)
    u = (iu - (g.nu - 1) / 2.0) * g.du
    if g.kind == 1:
        v = (iv - (g.nv - 1) / 2.0) * g.dv
        S = np.stack([g.sod * c, g.sod * sn, np.zeros_like(c)], axis=1)
        centre = -(g.sdd - g.sod) * np.stack([c, sn, np.zeros_like(c)], axis=1)
        eu = np.stack([-sn, c, np.zeros_like(c)], axis=1)
        ev = np.array([0.0, 0.0, 1.0])[None, :]
        P = centre + u[:, None] * eu + v[:, None] * ev
        d = P - S
    else:
        eu = np.stack([c, sn, np.zeros_like(c)], axis=1)
        S = u[:, None] * eu
        d = np.stack([-sn, c, np.zeros_like(c)], axis=1)
    d = d / np.linalg.norm(d, axis=1, keepdims=True)
    return S, d


def ellipsoid_line_integrals(g, ells, rays=None):
    """Sum over ellipsoids of density x chord length for each ray."""
    S, d = ray_geometry(g, rays)
    out = np.zeros(S.shape[0])
    for e in ells:
        Minv = (e.rot / e.semi[None, :]).T        # maps world offsets to the unit-sphere frame
        p0 = (S - e.centre[None, :]) @ Minv.T
        q = d @ Minv.T
        qq = np.einsum("ij,ij->i", q, q)
        pq = np.einsum("ij,ij->i", p0, q)
        pp = np.einsum("ij,ij->i", p0, p0)
        disc = pq * pq - qq * (pp - 1.0)
        chord = np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / qq, 0.0)
        out += e.density * chord
    return out

"""Seeded planet-shaped tetrahedral meshes (synthetic inputs only).

This module produces the *input* to the eigensolver: vertex coordinates,
linear tetrahedra and a per-tet region tag. It contains none of the
method's arithmetic (no shape functions, no integrals, no operators) and is
shared, as an input generator, by the CPU oracle and the GPU path.

Geometry (paper Sec. 2.1 builds its meshes from triangulated interfaces
and fills the volume with tetrahedra). Here every interface and the free
surface is an exact sphere, triangulated as a geodesic icosphere. The
volume between consecutive spheres is filled layer by layer:

* equal refinement level on both spheres: each triangular prism is split
  into three tetrahedra with the diagonal of every quadrilateral side face
  running from the lower vertex id of the inner sphere to the higher id of
  the outer one. The choice depends only on the edge, so neighbouring
  prisms always agree (conforming);
* the outer sphere one level finer: a fixed 7-tet template per coarse
  triangle (three corner tets and a split octahedron); the side faces are
  split symmetrically, so neighbours agree as well;
* the innermost sphere is a level-0 icosahedron coned to the centre.

Delaunay tetrahedralisation of shell points was tried first and produces
near-flat slivers (volume/edge^3 down to 1e-3) that inflate the top of
the stiffness spectrum by orders of magnitude; the layered construction
has no slivers. Seeded jitter (tangential everywhere, radial off the
interfaces) and a seeded global rotation make the mesh irregular.
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Mesh:
    xyz: np.ndarray      # (nv, 3) float64
    tet: np.ndarray      # (nt, 4) int32, positively oriented
    region: np.ndarray   # (nt,) uint8: 0 = solid, 1 = fluid
    layer: np.ndarray    # (nt,) int32: index of the radial layer (0 = innermost)
    radii: tuple         # interface radii, innermost first, last = surface

    @property
    def nv(self):
        return self.xyz.shape[0]

    @property
    def nt(self):
        return self.tet.shape[0]


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], float)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], np.int64)
    return v, f


def icosphere_levels(max_level):
    """Nested icosphere triangulations.

    Returns (verts, faces, mids): verts is the vertex array of the finest
    level (coarser levels use a prefix of it), faces[l] the triangles of
    level l, and mids[l] (for l < max_level) an array (nf_l, 3) with the
    midpoint vertex ids of edges (b,c), (c,a), (a,b) of each level-l face.
    """
    v, f = _icosahedron()
    verts = [v]
    nvert = len(v)
    faces = [f]
    mids = []
    for _ in range(max_level):
        edge_mid = {}
        new_pts = []

        def mid(a, b):
            nonlocal nvert
            key = (a, b) if a < b else (b, a)
            m = edge_mid.get(key)
            if m is None:
                m = nvert
                nvert += 1
                edge_mid[key] = m
                new_pts.append(key)
            return m

        fm = np.empty((len(f), 3), np.int64)
        for i, (a, b, c) in enumerate(f):
            fm[i] = (mid(b, c), mid(c, a), mid(a, b))
        allv = np.concatenate(verts)
        p = np.array([(allv[a] + allv[b]) * 0.5 for a, b in new_pts])
        p /= np.linalg.norm(p, axis=1, keepdims=True)
        verts.append(p)
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        mbc, mca, mab = fm[:, 0], fm[:, 1], fm[:, 2]
        nf = np.concatenate([np.stack([a, mab, mca], 1), np.stack([b, mbc, mab], 1),
                             np.stack([c, mca, mbc], 1), np.stack([mab, mbc, mca], 1)])
        mids.append(fm)
        faces.append(nf)
        f = nf
    return np.concatenate(verts), faces, mids


def _n_verts(level):
    return 10 * 4 ** level + 2


def _plan_shells(radii, h, max_level):
    """Shell radii and icosphere levels, innermost first.

    Within each region [r_a, r_b] shells are spaced evenly at about h; the
    level of a shell is the smallest one whose geodesic edge (about
    1.1 r / 2^l) is <= 1.25 h, raised by at most one per shell.
    """
    r0 = min(h, 0.5 * radii[0])
    shells = [(r0, 0)]
    lo = r0
    for rb in radii:
        nlay = max(1, int(np.ceil((rb - lo) / h - 1e-9)))
        for k in range(1, nlay + 1):
            r = lo + (rb - lo) * k / nlay
            want = 0
            while 1.1 * r / 2 ** want > 1.25 * h and want < max_level:
                want += 1
            prev = shells[-1][1]
            lev = min(max(want, prev), prev + 1)
            shells.append((r if k < nlay else rb, lev))
        lo = rb
    return shells


def layered_ball(radii=(1.0,), h=0.3, fluid_layers=(), seed=0, jitter=0.05,
                 max_level=6):
    """Tetrahedral mesh of a ball with exact spherical interfaces.

    radii: interface radii (increasing; last is the surface).
    h: target edge length. fluid_layers: indices into radii of layers that
    are fluid (layer i spans radii[i-1]..radii[i], layer 0 starts at 0).
    """
    radii = tuple(float(r) for r in radii)
    shells = _plan_shells(radii, h, max_level)
    lmax = max(l for _, l in shells)
    sv, sfaces, smids = icosphere_levels(lmax)
    rng = np.random.default_rng(seed)

    pts = [np.zeros((1, 3))]
    offs = []
    shell_pts_r = []
    base = 1
    for r, l in shells:
        n = _n_verts(l)
        offs.append(base)
        pts.append(sv[:n] * r)
        shell_pts_r.append(r)
        base += n
    xyz = np.concatenate(pts)
    tets = []
    # core: icosahedron coned to the centre
    f0 = sfaces[0]
    tets.append(np.stack([np.zeros(len(f0), np.int64), offs[0] + f0[:, 0],
                          offs[0] + f0[:, 1], offs[0] + f0[:, 2]], 1))
    tet_r = [np.full(len(f0), 0.5 * shells[0][0])]
    for k in range(len(shells) - 1):
        (ri, li), (ro, lo_) = shells[k], shells[k + 1]
        oi, oo = offs[k], offs[k + 1]
        if lo_ == li:
            f = np.sort(sfaces[li], axis=1)
            a, b, c = f[:, 0], f[:, 1], f[:, 2]
            t = np.concatenate([
                np.stack([oi + a, oi + b, oi + c, oo + c], 1),
                np.stack([oi + a, oi + b, oo + b, oo + c], 1),
                np.stack([oi + a, oo + a, oo + b, oo + c], 1)])
        else:
            f = sfaces[li]
            m = smids[li]
            A, B, C = f[:, 0], f[:, 1], f[:, 2]
            mbc, mca, mab = m[:, 0], m[:, 1], m[:, 2]
            t = np.concatenate([
                np.stack([oi + A, oo + A, oo + mab, oo + mca], 1),
                np.stack([oi + B, oo + B, oo + mbc, oo + mab], 1),
                np.stack([oi + C, oo + C, oo + mca, oo + mbc], 1),
                np.stack([oi + A, oo + mbc, oi + B, oi + C], 1),
                np.stack([oi + A, oo + mbc, oi + C, oo + mca], 1),
                np.stack([oi + A, oo + mbc, oo + mca, oo + mab], 1),
                np.stack([oi + A, oo + mbc, oo + mab, oi + B], 1)])
        tets.append(t)
        tet_r.append(np.full(len(t), 0.5 * (ri + ro)))
    tet = np.concatenate(tets)
    rmid = np.concatenate(tet_r)

    # seeded jitter: tangential for every shell vertex, radial only off the
    # interfaces; amplitude relative to the local edge length
    is_iface = np.zeros(len(xyz), bool)
    loc_h = np.zeros(len(xyz))
    for k, (r, l) in enumerate(shells):
        n = _n_verts(l)
        sl = slice(offs[k], offs[k] + n)
        loc_h[sl] = min(1.1 * r / 2 ** l, h)
        if any(abs(r - R) < 1e-12 for R in radii):
            is_iface[sl] = True
    rr = np.linalg.norm(xyz, axis=1)
    nz = rr > 0
    d = rng.normal(size=xyz.shape) * (jitter * loc_h)[:, None]
    u = np.zeros_like(xyz)
    u[nz] = xyz[nz] / rr[nz, None]
    d_rad = np.einsum('ij,ij->i', d, u)
    d_tan = d - d_rad[:, None] * u
    new = xyz + d_tan
    keep_r = np.where(is_iface, rr, rr + 0.5 * d_rad)
    nn = np.linalg.norm(new, axis=1)
    new[nz] *= (keep_r[nz] / nn[nz])[:, None]
    xyz = new

    # seeded global rotation
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, dd = q
    R = np.array([[a*a+b*b-c*c-dd*dd, 2*(b*c-a*dd), 2*(b*dd+a*c)],
                  [2*(b*c+a*dd), a*a-b*b+c*c-dd*dd, 2*(c*dd-a*b)],
                  [2*(b*dd-a*c), 2*(c*dd+a*b), a*a-b*b-c*c+dd*dd]])
    xyz = xyz @ R.T

    # positive orientation
    v = xyz[tet]
    vol = np.einsum('ij,ij->i', np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]),
                    v[:, 3] - v[:, 0])
    neg = vol < 0
    tet[neg, 2], tet[neg, 3] = tet[neg, 3].copy(), tet[neg, 2].copy()

    layer = np.searchsorted(np.asarray(radii), rmid).astype(np.int32)
    region = np.isin(layer, np.asarray(fluid_layers, int)).astype(np.uint8)
    return Mesh(xyz=np.ascontiguousarray(xyz, np.float64),
                tet=np.ascontiguousarray(tet, np.int32),
                region=region, layer=layer, radii=radii)


def tet_quality(xyz, tet):
    """6*sqrt(2)*volume / max_edge^3 (1 for a regular tet)."""
    v = xyz[tet]
    vol = np.einsum('ij,ij->i', np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]),
                    v[:, 3] - v[:, 0]) / 6.0
    e = np.stack([np.linalg.norm(v[:, i] - v[:, j], axis=1)
                  for i, j in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))], 1)
    return vol / e.max(1) ** 3 * 6 * np.sqrt(2)

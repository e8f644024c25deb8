"""CPU oracle: the self-gravitation term -C^T S C of the full operator.

Test infrastructure (CPU oracle). The perturbation S(u) of the
gravitational potential (paper Sec. 5.2, eqs. ph1body2, ph1surface2,
phi1fluidsolid, eigfull; Table matrixcomponentsselfG) is computed from
point masses at element and boundary-face barycentres:

  charge of element k:   q_k(u) = int_K div(rho_k u) dx = rho_k int_K div u dx
  charge of face l:      q_l(u) = int_E (nu . u) [rho]^+_- dS   on the outer
                         boundary (nu outward, [rho] = -rho_inside) and, on a
                         fluid-solid face, (nu^{f->s} . u^s) rho_s +
                         (nu^{s->f} . u^f) rho_f (each side's own copy),
                         and on an interior face of one region
                         (rho_+ - rho_-) (nu . u), nu from - to +;
  potential at point i:  S_i = G sum_{j != i} q_j / |r_i - r_j| + G q_i / R_i
  self distance:         1/R_i = (1/|K_i|) int_{K_i} dx / |r_i - x|
                         (element) or (1/|E_i|) int_{E_i} dS / |r_i - x| (face)
  form:                  a_G(u, v) = -sum_i q_i(v) S_i(u) = -(C v)^T S (C u),

so the full operator is K_eff - C^T S C. Reading taken where the paper is
silent on piecewise-constant densities: the density is the per-element
constant (its sampling of the model), so div(rho u) also has a surface
part on every interior face across which that constant jumps; those faces
(the paper's solid-solid and fluid-fluid discontinuities, Table
matrixcomponentsselfG) are charged with [rho]^+_- (nu . u), nu pointing
from the minus to the plus side, besides the outer boundary and the
fluid-solid faces. The charges of any displacement then sum to zero
(conservation of mass) for any per-element density.

With P2 shape functions the element charge involves only the edge nodes,
int_K d_i (4 l_a l_b) dx = |K| (d_i l_a + d_i l_b), the vertex functions
integrating to zero; on a face, int_E phi dS = |E|/3 for the edge nodes and
0 for the vertices.

The self distances are integrated here by splitting the element (face) into
cones from the barycentre over its faces (edges): int_K dx/|x - p| =
sum_faces (h_F / 2) int_F dS/|y - p| with the closed form of the triangle
integral, and int_E dS/|x - p| = sum_edges h_e int_e dl/|y - p| with the
closed form of the segment integral.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sps

from . import fem, p2

_TET_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))   # face opposite vertex i


def _tri_inv_dist(tri, p):
    """int over the triangle tri (3, 3) of dS / |y - p| in closed form.

    With h the signed height of p over the triangle's plane and, for each
    edge, t0 the in-plane distance from the foot of p to the edge line
    (positive when the foot is on the triangle's side), s-/s+ the edge
    end coordinates along the edge measured from the foot's projection,
    R-/R+ the distances from p to the ends and R0^2 = t0^2 + h^2:
      int dS/|y - p| = sum_edges t0 ln((R+ + s+) / (R- + s-))
                       - |h| sum_edges [atan(t0 s+ / (R0^2 + |h| R+))
                                        - atan(t0 s- / (R0^2 + |h| R-))]
    (the potential of a uniform triangle, Wilton et al. 1984)."""
    a, b, c = (np.asarray(x, np.float64) for x in tri)
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n)
    h = float(np.dot(p - a, n))
    ah = abs(h)
    foot = p - h * n
    total = 0.0
    verts = (a, b, c)
    centroid = (a + b + c) / 3.0
    for i in range(3):
        v0, v1 = verts[i], verts[(i + 1) % 3]
        L = v1 - v0
        l = L / np.linalg.norm(L)
        u = np.cross(l, n)                       # in-plane normal of the edge
        if np.dot(centroid - v0, u) > 0:         # make u point away from the triangle
            u = -u
        t0 = float(np.dot(v0 - foot, u))
        sm = float(np.dot(v0 - foot, l))
        sp = float(np.dot(v1 - foot, l))
        Rm = float(np.linalg.norm(v0 - p))
        Rp = float(np.linalg.norm(v1 - p))
        R02 = t0 * t0 + h * h
        if abs(t0) > 0.0:
            total += t0 * np.log((Rp + sp) / (Rm + sm))
            total -= ah * (np.arctan(t0 * sp / (R02 + ah * Rp)) - np.arctan(t0 * sm / (R02 + ah * Rm)))
    return total


def _segment_inv_dist(a, b, p):
    """int over the segment [a, b] of dl / |y - p| (closed form)."""
    L = np.linalg.norm(b - a)
    e = (b - a) / L
    ra, rb = np.linalg.norm(a - p), np.linalg.norm(b - p)
    ta, tb = np.dot(a - p, e), np.dot(b - p, e)
    return np.log((rb + tb) / (ra + ta))


def element_inv_R(xyz, tet):
    """1/R_k = (1/|K|) int_K dx / |x - r_k| for every tet (r_k the barycentre)."""
    vol, _ = p2.tet_geometry(xyz, tet)
    out = np.empty(len(tet))
    for k, t in enumerate(tet):
        v = xyz[t]
        r = v.mean(axis=0)
        s = 0.0
        for f in _TET_FACES:
            T = v[list(f)]
            nrm = np.cross(T[1] - T[0], T[2] - T[0])
            h = abs(np.dot(r - T[0], nrm)) / np.linalg.norm(nrm)
            s += 0.5 * h * _tri_inv_dist(T, r)
        out[k] = s / vol[k]
    return out


def face_inv_R(tri_xyz):
    """1/R_l = (1/|E|) int_E dS / |x - r_l| for triangles (nf, 3, 3)."""
    out = np.empty(len(tri_xyz))
    for l, T in enumerate(tri_xyz):
        r = T.mean(axis=0)
        area = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
        s = 0.0
        for i, j in ((0, 1), (1, 2), (2, 0)):
            a, b = T[i], T[j]
            e = (b - a) / np.linalg.norm(b - a)
            d = (r - a) - np.dot(r - a, e) * e
            s += np.linalg.norm(d) * _segment_inv_dist(a, b, r)
        out[l] = s / area
    return out


def _outer_faces(tet):
    """Faces owned by one tet only: (tet index, local face (3 vertex ids in
    the tet's order), opposite vertex id)."""
    tet = np.asarray(tet, np.int64)
    nt = len(tet)
    fv = np.concatenate([tet[:, list(f)] for f in _TET_FACES])
    owner = np.tile(np.arange(nt), 4)
    opp = np.repeat(np.arange(4), nt)
    key = np.sort(fv, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    one = cnt[inv.ravel()] == 1
    return owner[one], fv[one], tet[owner[one], opp[one]]


def _jump_faces(tet, region, rho):
    """Faces shared by two tets of one region whose densities differ:
    (minus tet, plus tet, face vertex ids in the minus tet's order,
    the minus tet's vertex opposite the face)."""
    tet = np.asarray(tet, np.int64)
    nt = len(tet)
    fv = np.concatenate([tet[:, list(f)] for f in _TET_FACES])
    owner = np.tile(np.arange(nt), 4)
    opp = np.repeat(np.arange(4), nt)
    key = np.sort(fv, axis=1)
    order = np.lexsort(key.T[::-1])
    ks = key[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    i0, i1 = order[:-1][same], order[1:][same]
    t0, t1 = owner[i0], owner[i1]
    keep = (region[t0] == region[t1]) & (rho[t0] != rho[t1])
    i0, t0, t1 = i0[keep], t0[keep], t1[keep]
    return t0, t1, fv[i0], tet[t0, opp[i0]]


def _edge_id(dm, nv, a, b):
    """P2 id of the edge (a, b)."""
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keys = dm.edges[:, 0] * (nv + 1) + dm.edges[:, 1]
    return nv + np.searchsorted(keys, lo * (nv + 1) + hi)


def charges(mesh, model):
    """Charge points (np, 3), inverse self distances (np,) and the charge
    matrix C (np x n, sparse) of the mesh's elements and charged faces."""
    xyz = np.asarray(mesh.xyz, np.float64)
    tet = np.asarray(mesh.tet, np.int64)
    region = np.asarray(mesh.region)
    nv = len(xyz)
    rho = np.asarray(model.rho, np.float64)
    dm = fem.dof_map(tet, region, nv)
    n = 3 * dm.Nu
    un = dm.elem_unodes(region)                       # (nt, 10) u-nodes
    vol, grads = p2.tet_geometry(xyz, tet)
    rows, cols, vals = [], [], []
    nt = len(tet)
    # elements: q_k = rho_k |K| sum_edges (grad l_a + grad l_b) . u_edge
    for e, (a, b) in enumerate(p2.EDGES):
        coef = (rho * vol)[:, None] * (grads[:, a] + grads[:, b])      # (nt, 3)
        node = un[:, 4 + e]
        for c in range(3):
            rows.append(np.arange(nt))
            cols.append(3 * node + c)
            vals.append(coef[:, c])
    points = [xyz[tet].mean(axis=1)]
    inv_R = [element_inv_R(xyz, tet)]
    base = nt
    # outer boundary faces: [rho] = -rho_inside, nu outward
    ot, otri, oppv = _outer_faces(tet)
    if len(ot):
        area, nrm = p2.face_geometry(xyz, otri)
        flip = np.einsum('ij,ij->i', xyz[oppv] - xyz[otri[:, 0]], nrm) > 0
        nrm[flip] *= -1.0
        for i, j in p2.FACE_EDGES:
            q = _edge_id(dm, nv, otri[:, i], otri[:, j])
            node = np.where(region[ot] == fem.SOLID, dm.unode_solid[q], dm.unode_fluid[q])
            coef = (-rho[ot] * area / 3.0)[:, None] * nrm
            for c in range(3):
                rows.append(base + np.arange(len(ot)))
                cols.append(3 * node + c)
                vals.append(coef[:, c])
        points.append(xyz[otri].mean(axis=1))
        inv_R.append(face_inv_R(xyz[otri]))
        base += len(ot)
    # interior faces of one region across which the per-element density
    # jumps: (rho_+ - rho_-) (nu . u), nu from the minus to the plus tet
    tm, tp, jtri, jopp = _jump_faces(tet, region, rho)
    if len(tm):
        area, nrm = p2.face_geometry(xyz, jtri)
        flip = np.einsum('ij,ij->i', xyz[jopp] - xyz[jtri[:, 0]], nrm) > 0
        nrm[flip] *= -1.0
        for i, j in p2.FACE_EDGES:
            q = _edge_id(dm, nv, jtri[:, i], jtri[:, j])
            node = np.where(region[tm] == fem.SOLID, dm.unode_solid[q], dm.unode_fluid[q])
            coef = ((rho[tp] - rho[tm]) * area / 3.0)[:, None] * nrm
            for c in range(3):
                rows.append(base + np.arange(len(tm)))
                cols.append(3 * node + c)
                vals.append(coef[:, c])
        points.append(xyz[jtri].mean(axis=1))
        inv_R.append(face_inv_R(xyz[jtri]))
        base += len(tm)
    # fluid-solid faces: rho_f (nu^{s->f} . u^f) - rho_s (nu^{s->f} . u^s)
    if dm.Np > 0 and (region == fem.SOLID).any():
        ts, tf, fn, nrm, area = fem.fs_faces(tet, dm.tet10, region, xyz)
        nf = len(ts)
        for k in range(3, 6):
            for node, dens in ((dm.unode_solid[fn[:, k]], -rho[ts]), (dm.unode_fluid[fn[:, k]], rho[tf])):
                coef = (dens * area / 3.0)[:, None] * nrm
                for c in range(3):
                    rows.append(base + np.arange(nf))
                    cols.append(3 * node + c)
                    vals.append(coef[:, c])
        tri = xyz[fn[:, :3]]
        points.append(tri.mean(axis=1))
        inv_R.append(face_inv_R(tri))
        base += nf
    C = sps.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(base, n)).tocsr()
    return np.concatenate(points), np.concatenate(inv_R), C


def kernel_matrix(points, inv_R, G):
    """S_ij = G / |r_i - r_j| (i != j), S_ii = G / R_i (dense)."""
    d = np.linalg.norm(points[:, None, :] - points[None, :, :], axis=2)
    np.fill_diagonal(d, 1.0)
    S = G / d
    np.fill_diagonal(S, G * inv_R)
    return S


def self_gravity_dense(mesh, model):
    """The dense matrix C^T S C (n x n) of the self-gravitation term."""
    pts, inv_R, C = charges(mesh, model)
    S = kernel_matrix(pts, inv_R, model.G)
    Cd = C.toarray()
    return Cd.T @ S @ Cd


def k_eff_full_dense(sys, mesh, model):
    """Dense K_eff - C^T S C (small problems)."""
    return fem.k_eff_dense(sys) - self_gravity_dense(mesh, model)

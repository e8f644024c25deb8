"""CPU oracle: P2 numbering and global assembly of the discrete pencil.

Test infrastructure: part of the CPU oracle; only tests, the smoke check
and the CPU-baseline leg of the benchmark use it. It shares no code with
the CUDA path.

Matrices (paper Sec. 4.2, Table of matrix formulae, and Appendix A), all
over the displacement nodes ("u-nodes") unless stated:

  M     = M_rho (x) I_3, M_rho = sum_k rho_k int phi_a phi_b        (b_H, mass)
  A_G   = blockdiag(A_sg, A_f)                                       (stiffness)
          A_sg: int grad v : c : grad u                         (solid tets)
                + S{ rho (div v)(g'.u) - rho u.(grad g').v
                     - rho u.(grad v).g' }                     (solid tets)
                + S{ (v.g')(nu_sf . u) rho_f }                  (FS faces)
          A_f : rho N^2 (g'.v)(g'.u)/|g'|^2                     (fluid tets)
  E_G   = [E_FS ; A_dg]  (u-dofs x p-nodes)
          E_FS: int_FS (v.nu_sf) p                              (FS faces)
          A_dg: int v.grad p - (v.g') p rho / kappa             (fluid tets)
  A_p   = -int p q / kappa                                      (fluid tets)
  R     = M_rho (x) [Omega]_x,   [Omega]_x u = Omega x u         (c_r)

and the Cowling operator K_eff = A_G - E_G A_p^{-1} E_G^T (Sec. 6.3,
eq. cowling). S{.} symmetrises a bilinear form (Sec. 2.2). The
coefficient rule follows Appendix A: rho, c, kappa, N^2 constant per tet;
g' and its element-local derivatives taken at the element nodes and
multiplied into the integrand as the P2 interpolant of the nodal product.
The reference field g' is computed by direct summation over tet point
masses at the barycentres (Sec. 5.1) with the Newtonian |x - r|^3 kernel.

Canonical numbering (an interface convention shared with the GPU library):
  P2 nodes: the mesh vertices 0..nv-1, then every edge once, in
    lexicographic order of (min vertex, max vertex), ids nv, nv+1, ...
  u-nodes: the P2 nodes touching a solid tet in increasing P2 id, then the
    P2 nodes touching a fluid tet in increasing P2 id (a node on a
    fluid-solid interface appears twice: a solid copy and a fluid copy).
  dof 3*u + c for component c of u-node u.
  p-nodes: the P2 nodes touching a fluid tet, in increasing P2 id.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sps

from . import p2

SOLID, FLUID = 0, 1
_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))   # face opposite vertex i


def p2_numbering(tet, nv):
    """P2 node ids per tet (nt, 10), number of P2 nodes, sorted edge list."""
    tet = np.asarray(tet, np.int64)
    e = np.concatenate([np.sort(tet[:, [i, j]], axis=1) for i, j in p2.EDGES])
    key = e[:, 0] * (nv + 1) + e[:, 1]
    uk, inv = np.unique(key, return_inverse=True)
    edges = np.stack([uk // (nv + 1), uk % (nv + 1)], 1)
    nt = len(tet)
    eid = inv.reshape(6, nt).T + nv
    return np.concatenate([tet, eid], axis=1), nv + len(uk), edges


def p2_coords(xyz, edges):
    return np.concatenate([xyz, 0.5 * (xyz[edges[:, 0]] + xyz[edges[:, 1]])])


@dataclasses.dataclass
class DofMap:
    tet10: np.ndarray     # (nt, 10) P2 ids
    n_p2: int
    edges: np.ndarray
    unode_solid: np.ndarray  # (n_p2,) u-node of the solid copy or -1
    unode_fluid: np.ndarray  # (n_p2,) u-node of the fluid copy or -1
    pnode: np.ndarray        # (n_p2,) p-node or -1
    Nu: int
    Np: int
    u_p2: np.ndarray         # (Nu,) P2 id of each u-node

    def elem_unodes(self, region):
        s = self.unode_solid[self.tet10]
        f = self.unode_fluid[self.tet10]
        return np.where((region == SOLID)[:, None], s, f)


def dof_map(tet, region, nv):
    tet10, n_p2, edges = p2_numbering(tet, nv)
    region = np.asarray(region)
    touch_s = np.zeros(n_p2, bool)
    touch_f = np.zeros(n_p2, bool)
    touch_s[tet10[region == SOLID].ravel()] = True
    touch_f[tet10[region == FLUID].ravel()] = True
    us = np.full(n_p2, -1, np.int64)
    uf = np.full(n_p2, -1, np.int64)
    ns = int(touch_s.sum())
    nf = int(touch_f.sum())
    us[touch_s] = np.arange(ns)
    uf[touch_f] = ns + np.arange(nf)
    pn = np.full(n_p2, -1, np.int64)
    pn[touch_f] = np.arange(nf)
    u_p2 = np.concatenate([np.nonzero(touch_s)[0], np.nonzero(touch_f)[0]])
    return DofMap(tet10, n_p2, edges, us, uf, pn, ns + nf, nf, u_p2)


def fs_faces(tet, tet10, region, xyz):
    """Faces shared by a solid and a fluid tet.

    Returns (solid_tet, fluid_tet, p2 ids (nf, 6) in face-local order,
    unit normal pointing from the solid into the fluid (nf, 3), area (nf,)).
    """
    tet = np.asarray(tet, np.int64)
    nt = len(tet)
    fv = np.concatenate([tet[:, list(f)] for f in _FACES])
    owner = np.tile(np.arange(nt), 4)
    opp = np.repeat(np.arange(4), nt)
    key = np.sort(fv, axis=1)
    order = np.lexsort(key.T[::-1])
    ks = key[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    i0 = order[:-1][same]
    i1 = order[1:][same]
    t0, t1 = owner[i0], owner[i1]
    r0, r1 = np.asarray(region)[t0], np.asarray(region)[t1]
    m = r0 != r1
    i0, i1, t0, t1, r0 = i0[m], i1[m], t0[m], t1[m], r0[m]
    si = np.where(r0 == SOLID, i0, i1)
    ts = np.where(r0 == SOLID, t0, t1)
    tf = np.where(r0 == SOLID, t1, t0)
    tri = fv[si]                               # vertex ids in the solid tet's order
    area, nrm = p2.face_geometry(xyz, tri)
    # orient the normal away from the solid tet's opposite vertex
    opp_v = tet[ts, opp[si]]
    d = np.einsum('ij,ij->i', xyz[opp_v] - xyz[tri[:, 0]], nrm)
    nrm[d > 0] *= -1.0
    # P2 ids of the face nodes: vertices, then edges (0,1), (0,2), (1,2)
    # located through the solid tet's local numbering
    loc = {}
    face_nodes = np.empty((len(tri), 6), np.int64)
    tv = tet[ts]
    t10 = tet10[ts]
    for k in range(3):
        face_nodes[:, k] = tri[:, k]
    edge_local = {e: 4 + i for i, e in enumerate(p2.EDGES)}
    for slot, (i, j) in enumerate(p2.FACE_EDGES):
        a = tri[:, i]
        b = tri[:, j]
        ids = np.empty(len(tri), np.int64)
        for (u, v), col in edge_local.items():
            hit = ((tv[:, u] == a) & (tv[:, v] == b)) | ((tv[:, u] == b) & (tv[:, v] == a))
            ids[hit] = t10[hit, col]
        face_nodes[:, 3 + slot] = ids
    del loc
    return ts, tf, face_nodes, nrm, area


def gravity_direct(points, xyz, tet, rho, G, chunk=2048, use_c=None):
    """g(x_i) = -G sum_k m_k (x_i - r_k) / |x_i - r_k|^3 (Sec. 5.1).

    m_k = rho_k |K_k|, r_k the barycentre of tet k. Large problems use the
    oracle's C loop (same formula, OpenMP over targets).
    """
    vol, _ = p2.tet_geometry(xyz, tet)
    m = np.asarray(rho) * vol
    rc = xyz[tet].mean(axis=1)
    if use_c is None:
        use_c = len(points) * len(tet) > 2e8
    if use_c:
        from . import cbuild
        lib = cbuild.load()
        src = np.ascontiguousarray(np.column_stack([rc, m]))
        pts = np.ascontiguousarray(points, np.float64)
        out = np.empty((len(points), 3))
        lib.oracle_gravity_direct(len(pts), pts.ctypes.data, len(src), src.ctypes.data, float(G),
                                  out.ctypes.data)
        return out
    out = np.empty((len(points), 3))
    for s in range(0, len(points), chunk):
        d = points[s:s + chunk, None, :] - rc[None, :, :]
        r2 = np.einsum('ijk,ijk->ij', d, d)
        w = m[None, :] / (r2 * np.sqrt(r2))
        out[s:s + chunk] = -G * np.einsum('ij,ijk->ik', w, d)
    return out


def _coo_blocks(rows, cols, vals, shape):
    return sps.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()


@dataclasses.dataclass
class System:
    dm: DofMap
    M_rho: sps.csr_matrix     # (Nu, Nu)
    M: sps.csr_matrix         # (n, n)
    A_G: sps.csr_matrix       # (n, n)
    E_G: sps.csr_matrix       # (n, Np)
    A_p: sps.csr_matrix       # (Np, Np)
    R: sps.csr_matrix         # (n, n)
    g_p2: np.ndarray          # (n_p2, 3) reference field at P2 nodes
    node_xyz: np.ndarray      # (n_p2, 3)

    @property
    def n(self):
        return 3 * self.dm.Nu

    def has_fluid(self):
        return self.dm.Np > 0


def assemble(mesh, model, gprime=None, chunk=20000):
    """Assemble every matrix of the pencil on the CPU (FP64)."""
    xyz = np.asarray(mesh.xyz, np.float64)
    tet = np.asarray(mesh.tet, np.int64)
    region = np.asarray(mesh.region)
    dm = dof_map(tet, region, len(xyz))
    node_xyz = p2_coords(xyz, dm.edges)
    Nu, Np = dm.Nu, dm.Np
    n = 3 * Nu
    rho = np.asarray(model.rho, np.float64)
    lam = np.asarray(model.lam, np.float64)
    mu = np.asarray(model.mu, np.float64)
    N2 = np.asarray(model.N2, np.float64)
    gravity = model.G != 0.0 or gprime is not None
    if gprime is not None:
        g = np.asarray(gprime, np.float64)
    elif model.G != 0.0:
        g = gravity_direct(node_xyz, xyz, tet, rho, model.G)
    else:
        g = np.zeros((dm.n_p2, 3))
    un = dm.elem_unodes(region)
    comp = np.arange(3)
    Mr = sps.csr_matrix((Nu, Nu))
    AG = sps.csr_matrix((n, n))
    EG = sps.csr_matrix((n, Np))
    Ap = sps.csr_matrix((Np, Np))
    for s in range(0, len(tet), chunk):
        sl = slice(s, s + chunk)
        t = tet[sl]
        vol, grads = p2.tet_geometry(xyz, t)
        r = rho[sl]
        Me = p2.mass_elem(vol)
        u = un[sl]
        Mr = Mr + _coo_blocks(np.repeat(u[:, :, None], 10, 2), np.repeat(u[:, None, :], 10, 1),
                              r[:, None, None] * Me, (Nu, Nu))
        dof = 3 * u[:, :, None] + comp[None, None, :]            # (nt, 10, 3)
        R5 = np.broadcast_to(dof[:, :, :, None, None], (len(t), 10, 3, 10, 3))
        C5 = np.broadcast_to(dof[:, None, None, :, :], (len(t), 10, 3, 10, 3))
        solid = region[sl] == SOLID
        fluid = ~solid
        Ke = p2.elastic_elem(vol, grads, lam[sl], mu[sl])
        Ke[fluid] = 0.0
        if gravity:
            ge = g[dm.tet10[sl]]                                  # (nt, 10, 3)
            C = p2.grad_val(vol, grads)                           # [t,a,p,b]
            dg = p2.nodal_grad(grads, ge)                         # [t,a,p,j]
            L = np.einsum('t,tamb,tbn->tambn', r, C, ge)
            L -= np.einsum('t,taij,tab->taibj', r, dg, Me)
            L -= np.einsum('t,tanb,tbm->tambn', r, C, ge)
            Ls = 0.5 * (L + np.transpose(L, (0, 3, 4, 1, 2)))
            Ls[fluid] = 0.0
            Ke += Ls
            # buoyancy in the fluid
            gn = np.linalg.norm(ge, axis=2, keepdims=True)
            gh = ge / np.where(gn > 0, gn, 1.0)
            Af = np.einsum('t,tai,tab,tbj->taibj', r * N2[sl], gh, Me, gh)
            Af[solid] = 0.0
            Ke += Af
        AG = AG + _coo_blocks(R5, C5, Ke, (n, n))
        if fluid.any():
            tf = np.nonzero(fluid)[0]
            kap = lam[sl][tf] + 2.0 * mu[sl][tf] / 3.0
            pn = dm.pnode[dm.tet10[sl][tf]]
            Ap = Ap + _coo_blocks(np.repeat(pn[:, :, None], 10, 2), np.repeat(pn[:, None, :], 10, 1),
                                  -(1.0 / kap)[:, None, None] * Me[tf], (Np, Np))
            Cf = p2.grad_val(vol[tf], grads[tf])                  # [t,b,j,a]
            Adg = np.transpose(Cf, (0, 3, 2, 1)).copy()           # [t,a,j,b]
            if gravity:
                ge_f = g[dm.tet10[sl][tf]]
                Adg -= np.einsum('t,taj,tab->tajb', r[tf] / kap, ge_f, Me[tf])
            dof_f = dof[tf]
            EG = EG + _coo_blocks(np.broadcast_to(dof_f[:, :, :, None], Adg.shape),
                                  np.broadcast_to(pn[:, None, None, :], Adg.shape), Adg, (n, Np))
    if Np > 0:
        ts, tf, fn, nrm, area = fs_faces(tet, dm.tet10, region, xyz)
        FM = area[:, None, None] * p2.FACE_MASS_REF[None]
        us = dm.unode_solid[fn]
        pn = dm.pnode[fn]
        dof_s = 3 * us[:, :, None] + comp[None, None, :]         # (nf, 6, 3)
        Efs = np.einsum('fab,fj->fajb', FM, nrm)
        EG = EG + _coo_blocks(np.broadcast_to(dof_s[:, :, :, None], Efs.shape),
                              np.broadcast_to(pn[:, None, None, :], Efs.shape), Efs, (n, Np))
        if gravity:
            gf = g[fn]
            rf = rho[tf]
            L = np.einsum('f,fam,fab,fn->fambn', rf, gf, FM, nrm)
            Ls = 0.5 * (L + np.transpose(L, (0, 3, 4, 1, 2)))
            AG = AG + _coo_blocks(np.broadcast_to(dof_s[:, :, :, None, None], Ls.shape),
                                  np.broadcast_to(dof_s[:, None, None, :, :], Ls.shape), Ls, (n, n))
    M = sps.kron(Mr, sps.identity(3), format='csr')
    Om = np.asarray(model.Omega, np.float64)
    W = np.array([[0, -Om[2], Om[1]], [Om[2], 0, -Om[0]], [-Om[1], Om[0], 0]])
    R = sps.kron(Mr, sps.csr_matrix(W), format='csr')
    return System(dm=dm, M_rho=Mr.tocsr(), M=M, A_G=AG.tocsr(), E_G=EG.tocsr(), A_p=Ap.tocsr(),
                  R=R, g_p2=g, node_xyz=node_xyz)


def k_eff_dense(sys: System):
    """Dense Cowling operator A_G - E_G A_p^{-1} E_G^T (small problems)."""
    K = sys.A_G.toarray()
    if sys.has_fluid():
        EG = sys.E_G.toarray()
        K = K - EG @ np.linalg.solve(sys.A_p.toarray(), EG.T)
    return 0.5 * (K + K.T)


def k_eff_apply(sys: System, X, tol=1e-14):
    """K_eff X with A_p^{-1} by a sparse direct solve."""
    Y = sys.A_G @ X
    if sys.has_fluid():
        import scipy.sparse.linalg as spla
        lu = spla.splu(sys.A_p.tocsc())
        Y = Y - sys.E_G @ lu.solve(np.asarray(sys.E_G.T @ X))
    return Y

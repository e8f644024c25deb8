"""P2 tetrahedral element integrals by exact barycentric integration.

Test infrastructure: this module is part of the CPU oracle. Only tests,
the smoke check and the CPU-baseline leg of the benchmark use it.

The paper builds its element matrices on a reference tetrahedron through a
generalized Vandermonde matrix (Appendix A: M = V^-T V^-1, D_j =
(d_r V) V^-1). The oracle reaches the same exact integrals by a different
route: quadratic Lagrange shape functions written in barycentric
coordinates,

    vertex i : l_i (2 l_i - 1),    edge (i,j) : 4 l_i l_j,

multiplied out as polynomials in (l_0, l_1, l_2, l_3) and integrated with

    int_K l^a dx = 3! a_0! a_1! a_2! a_3! |K| / (|a| + 3)!      (tetrahedron)
    int_F l^a ds = 2! a_0! a_1! a_2! |F| / (|a| + 2)!            (triangle)

Local node order: the 4 vertices, then the edges (0,1), (0,2), (0,3),
(1,2), (1,3), (2,3). On a face with vertices (0,1,2) the local order is the
3 vertices then edges (0,1), (0,2), (1,2).
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial
import itertools
import numpy as np

EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
FACE_EDGES = ((0, 1), (0, 2), (1, 2))


def _poly_mul(p, q):
    out = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return out


def _poly_diff(p, k):
    out = {}
    for e, c in p.items():
        if e[k] > 0:
            e2 = list(e)
            e2[k] -= 1
            out[tuple(e2)] = out.get(tuple(e2), 0) + c * e[k]
    return out


def _unit(nvar, k, power=1):
    e = [0] * nvar
    e[k] = power
    return tuple(e)


def shape_polys(nvar):
    """P2 shape functions as polynomials in nvar barycentric coordinates."""
    edges = EDGES if nvar == 4 else FACE_EDGES
    polys = []
    for i in range(nvar):
        polys.append({_unit(nvar, i, 2): Fraction(2), _unit(nvar, i, 1): Fraction(-1)})
    for i, j in edges:
        e = [0] * nvar
        e[i] = 1
        e[j] = 1
        polys.append({tuple(e): Fraction(4)})
    return polys


def _integrate(p, dim):
    """int l^a over a simplex of unit measure (dim = 3 tet, 2 triangle)."""
    s = Fraction(0)
    for e, c in p.items():
        num = factorial(dim)
        for a in e:
            num *= factorial(a)
        s += c * Fraction(num, factorial(sum(e) + dim))
    return s


def _eval(p, lam):
    s = Fraction(0)
    for e, c in p.items():
        t = c
        for a, l in zip(e, lam):
            t *= Fraction(l) ** a
        s += t
    return s


def _build_reference():
    phi = shape_polys(4)
    dphi = [[_poly_diff(p, k) for k in range(4)] for p in phi]
    mass = np.zeros((10, 10))
    cref = np.zeros((10, 4, 10))       # int (d phi_a / d l_k) phi_b
    sref = np.zeros((10, 4, 10, 4))    # int (d phi_a / d l_k)(d phi_b / d l_l)
    for a, b in itertools.product(range(10), range(10)):
        mass[a, b] = float(_integrate(_poly_mul(phi[a], phi[b]), 3))
        for k in range(4):
            cref[a, k, b] = float(_integrate(_poly_mul(dphi[a][k], phi[b]), 3))
            for l in range(4):
                sref[a, k, b, l] = float(_integrate(_poly_mul(dphi[a][k], dphi[b][l]), 3))
    # barycentric coordinates of the 10 local nodes
    nodes = [tuple(Fraction(int(i == k)) for k in range(4)) for i in range(4)]
    for i, j in EDGES:
        nodes.append(tuple(Fraction(1, 2) if k in (i, j) else Fraction(0) for k in range(4)))
    # dnode[c, k, a] = (d phi_c / d l_k) evaluated at node a
    dnode = np.zeros((10, 4, 10))
    for c, k, a in itertools.product(range(10), range(4), range(10)):
        dnode[c, k, a] = float(_eval(dphi[c][k], nodes[a]))
    fphi = shape_polys(3)
    fmass = np.zeros((6, 6))
    for a, b in itertools.product(range(6), range(6)):
        fmass[a, b] = float(_integrate(_poly_mul(fphi[a], fphi[b]), 2))
    return mass, cref, sref, dnode, fmass


MASS_REF, CREF, SREF, DNODE, FACE_MASS_REF = _build_reference()


def tet_geometry(xyz, tet):
    """Volumes (nt,) and barycentric gradients (nt, 4, 3) of linear tets."""
    v = xyz[tet]
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)           # rows: grad of l_1, l_2, l_3
    grads = np.empty((len(tet), 4, 3))
    grads[:, 1:, :] = Jinv
    grads[:, 0, :] = -Jinv.sum(axis=1)
    return np.abs(det) / 6.0, grads


def mass_elem(vol):
    """int phi_a phi_b over each tet: (nt, 10, 10)."""
    return vol[:, None, None] * MASS_REF[None]


def grad_grad(vol, grads):
    """D[t, a, p, b, q] = int d_p phi_a d_q phi_b: (nt, 10, 3, 10, 3)."""
    return np.einsum('t,akbl,tkp,tlq->tapbq', vol, SREF, grads, grads, optimize=True)


def grad_val(vol, grads):
    """C[t, a, p, b] = int (d_p phi_a) phi_b: (nt, 10, 3, 10)."""
    return np.einsum('t,akb,tkp->tapb', vol, CREF, grads, optimize=True)


def nodal_grad(grads, nodal):
    """Gradient of the element's P2 interpolant at its own nodes.

    nodal: (nt, 10, m) values at the element's nodes. Returns
    (nt, 10, 3, m): [t, a, p, j] = d_p (interpolant of component j) at node a.
    """
    return np.einsum('ckA,tkp,tcj->tApj', DNODE, grads, nodal, optimize=True)


def elastic_elem(vol, grads, lam, mu):
    """Isotropic elastic stiffness int grad v : c : grad u, (nt, 10, 3, 10, 3).

    c_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) (isotropic form of the
    stiffness tensor in the paper's Table of matrix formulae, solid rows).
    """
    D = grad_grad(vol, grads)
    lap = np.einsum('tapbp->tab', D)
    K = lam[:, None, None, None, None] * D
    K += mu[:, None, None, None, None] * np.transpose(D, (0, 1, 4, 3, 2))
    K += mu[:, None, None, None, None] * lap[:, :, None, :, None] * np.eye(3)[None, None, :, None, :]
    return K


def face_geometry(xyz, tri):
    """Areas (nf,) and unit normals (nf, 3) (right-hand rule) of triangles."""
    v = xyz[tri]
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    a = np.linalg.norm(n, axis=1)
    return 0.5 * a, n / a[:, None]

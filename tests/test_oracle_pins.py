"""Pins of the CPU oracle against closed forms, invariants and library routines.

Every check here is independent of the oracle's own arithmetic: exact
values a plain derivation gives, quadrature by another rule, dense or
sparse library eigensolvers, physics limits (Lamb, rigid cavity acoustics,
Newtonian gravity of a ball), so that a dropped term, a wrong sign or a
transposed operand in the oracle fails one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla
from scipy.special import spherical_jn
from scipy.optimize import brentq

from synth.mesh import layered_ball, tet_quality
from synth.model import Model, config_ball, homogeneous_ball, layered_planet
from oracle import p2, fem, eig, filtlan
from oracle.lamb import lamb_modes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ quadrature
def _duffy_rule(n):
    """Collapsed-cube Gauss rule on the unit tet {x,y,z >= 0, x+y+z <= 1}."""
    g, w = np.polynomial.legendre.leggauss(n)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    pts, wts = [], []
    for a, wa in zip(g, w):
        for b, wb in zip(g, w):
            for c, wc in zip(g, w):
                x = a
                y = b * (1 - a)
                z = c * (1 - a) * (1 - b)
                pts.append((x, y, z))
                wts.append(wa * wb * wc * (1 - a) ** 2 * (1 - b))
    return np.array(pts), np.array(wts)


def _p2_shape(lam):
    """P2 shape values at barycentric points (q, 4) -> (q, 10), by direct formula."""
    out = [lam[:, i] * (2 * lam[:, i] - 1) for i in range(4)]
    out += [4 * lam[:, i] * lam[:, j] for i, j in p2.EDGES]
    return np.stack(out, 1)


def test_reference_mass_by_quadrature():
    pts, wts = _duffy_rule(6)
    lam = np.column_stack([1 - pts.sum(1), pts])
    phi = _p2_shape(lam)
    Mq = np.einsum('q,qa,qb->ab', wts, phi, phi) / (1.0 / 6.0)   # per unit volume
    assert np.allclose(p2.MASS_REF, Mq, atol=1e-14)


def test_mass_row_sums_closed_form():
    # int phi_vertex = -|K|/20, int phi_edge = |K|/5 for P2 on a tet
    rs = p2.MASS_REF.sum(1)
    assert np.allclose(rs[:4], -1 / 20, atol=1e-15)
    assert np.allclose(rs[4:], 1 / 5, atol=1e-15)


def test_jacobi_mass_spectrum_closed_form():
    ev = np.sort(np.linalg.eigvals(np.diag(1 / np.diag(p2.MASS_REF)) @ p2.MASS_REF).real)
    assert abs(ev[0] - 0.25) < 1e-13
    assert abs(ev[-1] - (19 + np.sqrt(249.0)) / 8) < 1e-12
    assert filtlan.MASS_LO == 0.25 and abs(filtlan.MASS_HI - ev[-1]) < 1e-12


def test_grad_grad_by_quadrature_on_physical_tet():
    rng = np.random.default_rng(5)
    xyz = np.array([[0, 0, 0], [1.1, 0.1, 0], [0.2, 0.9, 0.1], [0.1, 0.3, 1.2]]) + rng.normal(0, 0.05, (4, 3))
    tet = np.array([[0, 1, 2, 3]])
    vol, grads = p2.tet_geometry(xyz, tet)
    D = p2.grad_grad(vol, grads)[0]
    C = p2.grad_val(vol, grads)[0]
    # quadrature of the shape-function gradients via finite differences of the
    # direct formula in physical coordinates (central, step 1e-5) and a Duffy rule
    pts, wts = _duffy_rule(5)
    J = np.stack([xyz[1] - xyz[0], xyz[2] - xyz[0], xyz[3] - xyz[0]], 1)
    X = xyz[0] + pts @ J.T
    Jinv = np.linalg.inv(J)

    def shape_at(x):
        r = (x - xyz[0]) @ Jinv.T
        return _p2_shape(np.column_stack([1 - r.sum(1), r]))

    h = 1e-5
    G = np.stack([(shape_at(X + h * e) - shape_at(X - h * e)) / (2 * h) for e in np.eye(3)], 2)
    phi = shape_at(X)
    detJ = abs(np.linalg.det(J))
    Dq = np.einsum('q,qap,qbr->apbr', wts * detJ, G, G)
    Cq = np.einsum('q,qap,qb->apb', wts * detJ, G, phi)
    assert np.allclose(D, Dq, atol=1e-8 * abs(D).max())
    assert np.allclose(C, Cq, atol=1e-8 * abs(C).max())


def test_nodal_grad_exact_for_quadratics():
    xyz = np.array([[0, 0, 0], [1.0, 0.2, 0], [0.1, 1.1, 0], [0.2, 0.1, 0.9]])
    tet10, _, edges = fem.p2_numbering(np.array([[0, 1, 2, 3]]), 4)
    nodes = fem.p2_coords(xyz, edges)[tet10[0]]
    f = lambda x: np.stack([x[:, 0] * x[:, 1], x[:, 2] ** 2, x[:, 0]], 1)     # quadratic field
    df = lambda x: np.stack([np.stack([x[:, 1], np.zeros(len(x)), np.ones(len(x))], 1),
                             np.stack([x[:, 0], np.zeros(len(x)), np.zeros(len(x))], 1),
                             np.stack([np.zeros(len(x)), 2 * x[:, 2], np.zeros(len(x))], 1)], 1)
    _, grads = p2.tet_geometry(xyz, np.array([[0, 1, 2, 3]]))
    g = p2.nodal_grad(grads, f(nodes)[None])[0]                # [a, p, j]
    assert np.allclose(g, df(nodes), atol=1e-12)


# ------------------------------------------------------------ mesh
def test_mesh_conforming_and_quality():
    m = layered_ball(radii=(0.19, 0.55, 1.0), h=0.12, fluid_layers=(1,), seed=4)
    assert tet_quality(m.xyz, m.tet).min() > 0.08
    f = np.sort(np.concatenate([m.tet[:, [1, 2, 3]], m.tet[:, [0, 2, 3]],
                                m.tet[:, [0, 1, 3]], m.tet[:, [0, 1, 2]]]), 1)
    _, cnt = np.unique(f, axis=0, return_counts=True)
    assert cnt.max() == 2
    # boundary faces lie on the unit sphere (vertices exactly on it)
    bf = np.unique(f, axis=0, return_counts=True)
    bverts = np.unique(bf[0][bf[1] == 1])
    assert np.allclose(np.linalg.norm(m.xyz[bverts], axis=1), 1.0, atol=1e-12)


# ------------------------------------------------------------ elastic ball
@pytest.fixture(scope="module")
def ball():
    w = config_ball()
    S = fem.assemble(w.mesh, w.model)
    K, M = eig.pencil_dense(S)
    lam, X = eig.all_eigs(K, M)
    return w, S, K, M, lam, X


def _rigid_modes(S):
    x = S.node_xyz[S.dm.u_p2]
    Nu = len(x)
    out = []
    for c in range(3):
        v = np.zeros((Nu, 3))
        v[:, c] = 1
        out.append(v.ravel())
    for axis in np.eye(3):
        out.append(np.cross(axis, x).ravel())
    return np.stack(out, 1)


def test_ball_matrices_symmetric_spd(ball):
    _, S, K, M, _, _ = ball
    assert abs(K - K.T).max() <= 1e-14 * abs(K).max()
    assert abs(M - M.T).max() <= 1e-15 * abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0
    # total mass: 1^T M_rho 1 = sum rho |K|
    vol, _ = p2.tet_geometry(w_xyz := ball[0].mesh.xyz, ball[0].mesh.tet)
    assert np.isclose(S.M_rho.sum(), (ball[0].model.rho * vol).sum(), rtol=1e-13)


def test_ball_rigid_null_space(ball):
    _, S, K, M, lam, X = ball
    Rm = _rigid_modes(S)
    assert np.abs(K @ Rm).max() <= 1e-12 * abs(K).max()
    lmax = lam[-1]
    zero = np.abs(lam) <= 1e-10 * lmax
    assert zero.sum() == 6
    # the zero eigenvectors span the rigid motions
    Q, _ = np.linalg.qr(Rm)
    Z = X[:, zero]
    resid = Z - Q @ (Q.T @ Z)
    assert np.linalg.norm(resid) <= 1e-8 * np.linalg.norm(Z)


def test_ball_slice_count_and_multiplets(ball):
    _, _, _, _, lam, _ = ball
    om = np.sqrt(np.clip(lam, 0, None))
    assert ((om >= 0) & (om <= 3.0)).sum() == 16
    # two 5-fold groups above the zero modes: 0T2 then 0S2
    t2 = om[6:11]
    s2 = om[11:16]
    assert t2.max() - t2.min() < 0.03 and s2.max() - s2.min() < 0.03
    assert t2.max() < s2.min()


def test_lamb_golden_matches_closed_form():
    with open(os.path.join(GOLDEN, "lamb_ball.json")) as f:
        g = json.load(f)
    modes = lamb_modes(6.0)
    assert [m[1] for m in modes] == [m["label"] for m in g["modes"]]
    assert np.allclose([m[0] for m in modes], [m["omega"] for m in g["modes"]], rtol=1e-12)


def test_lamb_toroidal_is_first_root_of_bessel_relation():
    # independent check of the toroidal relation: (l-1) j_l - x j_{l+1}
    # equals x^2 d/dx (j_l / x) (spherical-Bessel identity), so its roots are
    # the stationary points of j_l(x)/x
    f = lambda x: (spherical_jn(2, x + 1e-6) / (x + 1e-6) - spherical_jn(2, x - 1e-6) / (x - 1e-6))
    x0 = brentq(f, 1.0, 3.0)
    assert abs(x0 - lamb_modes(3.0)[0][0]) < 1e-6


def _traction_at_surface(l, kind, vp=1.7, vs=1.0, rho=1.0, th0=0.7):
    """Surface traction of Cartesian displacement fields built from potentials.

    A field independent of the radial functions in oracle/lamb.py: for a
    homogeneous ball the displacement is grad(phi) (P), curl curl(x psi)
    (S) or curl(x chi) (T) with phi, psi, chi = j_l(kappa r) P_l(cos theta)
    (Navier's equation holds for kappa = w / Vp or w / Vs); the traction
    sigma . r_hat at r = 1, theta = th0 is formed by symbolic Cartesian
    differentiation (sympy). Returns callables of w giving the (r, theta,
    phi) traction components for each field."""
    sp = pytest.importorskip("sympy")
    x, y, z, w = sp.symbols('x y z w', real=True)
    r = sp.sqrt(x * x + y * y + z * z)
    X = sp.Matrix([x, y, z])
    s = sp.Symbol('s')
    jl = sp.sin(s) / s
    for _ in range(l):
        jl = sp.diff(jl, s) / s
    jl = (-s) ** l * jl                     # Rayleigh's formula for j_l

    def pot(kk):
        return jl.subs(s, kk * r) * sp.legendre(l, z / r)

    def grad(f):
        return sp.Matrix([sp.diff(f, v) for v in (x, y, z)])

    def curl(F):
        return sp.Matrix([sp.diff(F[2], y) - sp.diff(F[1], z), sp.diff(F[0], z) - sp.diff(F[2], x),
                          sp.diff(F[1], x) - sp.diff(F[0], y)])

    mu = rho * vs * vs
    lam = rho * vp * vp - 2 * mu
    h, k = w / vp, w / vs
    fields = {"S": [grad(pot(h)), curl(curl(X * pot(k)))], "T": [curl(X * pot(k))], "R": [grad(pot(h))]}[kind]
    pt = {x: sp.sin(th0), y: 0, z: sp.cos(th0)}
    frame = (sp.Matrix([sp.sin(th0), 0, sp.cos(th0)]), sp.Matrix([sp.cos(th0), 0, -sp.sin(th0)]),
             sp.Matrix([0, 1, 0]))
    out = []
    for u in fields:
        J = u.jacobian(X)
        sig = lam * J.trace() * sp.eye(3) + mu * (J + J.T)
        t = (sig * X / r).subs(pt)
        out.append([sp.lambdify(w, (t.T * e)[0], 'mpmath') for e in frame])
    return out


def test_lamb_modes_from_independent_potential_fields():
    """The closed-form Lamb frequencies (oracle/lamb.py, radial functions U,
    V) are roots of the traction-free condition formed from 3-D Cartesian
    potential fields instead: the 2 x 2 traction determinant of the P and S
    fields (spheroidal), the phi traction of the T field (toroidal) and the
    radial traction of the P field (l = 0)."""
    import mpmath
    mpmath.mp.dps = 30
    modes = {lab: om for om, lab, _ in lamb_modes(6.0)}
    for lab, l, kind in (("0T2", 2, "T"), ("0S2", 2, "S"), ("1S1", 1, "S"), ("0S0", 0, "R"), ("0T3", 3, "T"),
                         ("1S2", 2, "S")):
        f = _traction_at_surface(l, kind)
        if kind == "S":
            g = lambda w: float(f[0][0](w) * f[1][1](w) - f[1][0](w) * f[0][1](w))
        elif kind == "T":
            g = lambda w: float(f[0][2](w))
        else:
            g = lambda w: float(f[0][0](w))
        root = brentq(g, modes[lab] - 0.03, modes[lab] + 0.03, xtol=1e-14)
        assert root == pytest.approx(modes[lab], rel=1e-12), lab


def test_ball_converges_to_lamb():
    """0T2 and 0S2 multiplet means approach Lamb's values under refinement."""
    exact = {m[1]: m[0] for m in lamb_modes(3.0)}
    errs = []
    for h in (0.45, 0.3):
        mesh, model = homogeneous_ball(h=h, seed=1)
        S = fem.assemble(mesh, model)
        w, _ = eig.eigs_near(S, 2.55 ** 2, 16)
        om = np.sort(np.sqrt(np.clip(w, 0, None)))
        om = om[om > 1.0][:10]
        errs.append((om[:5].mean() / exact["0T2"] - 1, om[5:].mean() / exact["0S2"] - 1))
    (t0, s0), (t1, s1) = errs
    assert 0 < t1 < t0 < 0.06 and 0 < s1 < s0 < 0.06
    assert t1 < 0.02 and s1 < 0.02


# ------------------------------------------------------------ fluid pieces
def _fluid_ball(h, vp=1.3, rho=1.0):
    m = layered_ball(radii=(1.0,), h=h, fluid_layers=(0,), seed=3)
    nt = m.nt
    mdl = Model(rho=np.full(nt, rho), lam=np.full(nt, rho * vp * vp), mu=np.zeros(nt),
                N2=np.zeros(nt), G=0.0, Omega=np.zeros(3))
    return fem.assemble(m, mdl), vp


def test_fluid_ball_rigid_cavity_acoustics():
    """A fluid ball without gravity is a rigid-walled acoustic cavity.

    The weak pressure constraint without a free-surface term imposes
    u.nu = 0 on the boundary, so the nonzero modes tend to
    omega = Vp x with j_l'(x) = 0 (l = 1: x = 2.0816, l = 2: 3.3421).
    """
    S, vp = _fluid_ball(0.3)
    w, _ = eig.eigs_near(S, (2.7 * vp) ** 2, 12)
    x = np.sqrt(np.clip(w, 0, None)) / vp
    x = np.sort(x[x > 1.0])
    r1 = brentq(lambda t: spherical_jn(1, t, derivative=True), 1.5, 2.5)
    r2 = brentq(lambda t: spherical_jn(2, t, derivative=True), 3.0, 3.6)
    assert np.allclose(x[:3], r1, rtol=0.02) and (x[:3] > r1).all()
    assert np.allclose(x[3:8], r2, rtol=0.02) and (x[3:8] > r2).all()


def test_fluid_pressure_blocks_closed_forms():
    S, vp = _fluid_ball(0.45)
    kap = vp * vp
    vol = S.M_rho.sum()          # rho = 1
    assert np.isclose(S.A_p.sum(), -vol / kap, rtol=1e-12)
    # A_dg: int v.grad p for v = e_j and p = a.x (exact in P2)
    a = np.array([0.3, -1.2, 0.7])
    p = S.node_xyz[np.nonzero(S.dm.pnode >= 0)[0]] @ a
    for j in range(3):
        v = np.zeros(S.n)
        v[j::3] = 1.0
        assert np.isclose(v @ (S.E_G @ p), a[j] * vol, rtol=1e-12)


def test_layered_rigid_modes_without_gravity():
    """Solid-fluid-solid ball without gravity: the 6 rigid motions stay exact
    zero modes of K_eff, which needs E_FS and A_dg with consistent signs
    (the fluid-side and solid-side boundary integrals cancel)."""
    mesh, model = layered_planet(h=0.25, seed=7)
    model.G = 0.0
    S = fem.assemble(mesh, model)
    Rm = _rigid_modes(S)
    assert np.abs(S.E_G.T @ Rm).max() <= 1e-12 * abs(S.E_G).max()
    K = fem.k_eff_dense(S)
    assert np.abs(K @ Rm).max() <= 1e-10 * abs(K).max()
    # and E_FS alone does not vanish on them (the cancellation is real)
    fs_rows = np.zeros(S.n, bool)
    fs_rows[:3 * int((S.dm.unode_solid >= 0).sum())] = True
    assert np.abs(S.E_G[fs_rows].T @ Rm[fs_rows]).max() > 1e-3


def test_cowling_homogeneous_ball_rigid_motions():
    """Cowling approximation (reference field fixed, no S(u)): a homogeneous
    ball translated rigidly oscillates in its own potential well with
    omega^2 = (4/3) pi G rho, and rigid rotations cost no energy. This pins
    the signs and weights of all three symmetrised gravity volume terms."""
    mesh, model = homogeneous_ball(h=0.3, seed=1)
    model.G = 1.0 / np.pi
    S = fem.assemble(mesh, model)
    K = fem.k_eff_dense(S)
    M = S.M.toarray()
    Rm = _rigid_modes(S)
    ray = np.diag(Rm.T @ K @ Rm) / np.diag(Rm.T @ M @ Rm)
    assert np.allclose(ray[:3], 4.0 / 3.0 * np.pi * model.G * 1.0, rtol=0.01)
    assert np.abs(ray[3:]).max() < 0.01
    lam = eig.all_eigs(K, M)[0]
    assert np.allclose(lam[3:6], 4.0 / 3.0, rtol=0.01)


def test_layered_cowling_spectrum_structure():
    """Three-layer planet, Cowling: K_eff symmetric; the only clearly
    negative modes are three near-rigid rotations of the inner core
    (rigid rotations in a radial field cost nothing; the direct-summation
    field's non-radial error on the coarse 0.19-radius core makes them
    slightly negative, and it shrinks under refinement, see below); a large
    near-zero cluster comes from the fluid (essential spectrum)."""
    mesh, model = layered_planet(h=0.25, seed=7)
    S = fem.assemble(mesh, model)
    assert abs(S.A_G - S.A_G.T).max() <= 1e-13 * abs(S.A_G).max()
    K = fem.k_eff_dense(S)
    M = S.M.toarray()
    lam, X = eig.all_eigs(K, M)
    neg = np.nonzero(lam < -0.01)[0]
    assert len(neg) == 3
    ns = int((S.dm.unode_solid >= 0).sum())
    x = S.node_xyz[S.dm.u_p2]
    ic = (np.linalg.norm(x, axis=1) < 0.19 + 1e-9) & (np.arange(len(x)) < ns)
    rot = []
    for axis in np.eye(3):
        u = np.zeros((len(x), 3))
        u[ic] = np.cross(axis, x[ic])
        rot.append(u.ravel())
    rot = np.stack(rot, 1)
    for i in neg:
        v = X[:, i]
        r = v - rot @ np.linalg.lstsq(rot, v, rcond=None)[0]
        assert r @ M @ r <= 0.01 * (v @ M @ v)
    assert (np.abs(lam) < 0.01).sum() > 0.2 * S.dm.Np


def test_layered_rigid_rotations_cost_nothing_under_refinement():
    """Rigid rotations of a spherically symmetric planet in its own radial
    reference field are zero-energy motions of K_eff (Sec. 2.3: no strain,
    u.g' = 0, and the gravity derivative terms cancel). With the
    direct-summation field of a polyhedral mesh their Rayleigh quotients,
    small against the gravity scale (4/3) pi G rho ~ 1.3, fall under
    refinement: for the whole planet (K_eff) and for the inner core alone
    (A_G: the solid and interface gravity terms)."""
    out = []
    for h in (0.25, 0.15):
        mesh, model = layered_planet(h=h, seed=7)
        S = fem.assemble(mesh, model)
        ns = int((S.dm.unode_solid >= 0).sum())
        x = S.node_xyz[S.dm.u_p2]
        ic = (np.linalg.norm(x, axis=1) < 0.19 + 1e-9) & (np.arange(len(x)) < ns)
        whole, core = [], []
        for axis in np.eye(3):
            u = np.cross(axis, x).ravel()
            whole.append(abs(u @ fem.k_eff_apply(S, u[:, None]).ravel()) / (u @ (S.M @ u)))
            v = np.zeros((len(x), 3))
            v[ic] = np.cross(axis, x[ic])
            v = v.ravel()
            core.append(abs(v @ (S.A_G @ v)) / (v @ (S.M @ v)))
        out.append((max(whole), max(core)))
    (w0, c0), (w1, c1) = out
    assert w1 < w0 < 5e-3
    assert c1 < 0.1 * c0 and c1 < 0.01


def test_gravity_direct_summation_homogeneous_ball():
    """Point-mass direct summation (Sec. 5.1) against Newton for a ball.

    Outside: the monopole -G M x/|x|^3 to 5e-4. Inside the field is
    -(4/3) pi G rho x; point masses at the barycentres carry an O(h)
    pointwise error from the nearest masses, so the pin is the radially
    averaged interior field (a few per cent) and its decrease under
    refinement.
    """
    G = 1.0 / np.pi
    far = np.array([[2.0, 0.0, 0.0], [0.0, -3.0, 1.0]])
    errs = []
    for h in (0.3, 0.2):
        mesh, model = homogeneous_ball(h=h, seed=1)
        vol, _ = p2.tet_geometry(mesh.xyz, mesh.tet)
        Mtot = vol.sum()
        gf = fem.gravity_direct(far, mesh.xyz, mesh.tet, model.rho, G)
        ex = -G * Mtot * far / np.linalg.norm(far, axis=1, keepdims=True) ** 3
        assert np.abs(gf - ex).max() <= 5e-4 * np.abs(ex).max()
        x = mesh.xyz[np.linalg.norm(mesh.xyz, axis=1) < 0.8]
        x = x[np.linalg.norm(x, axis=1) > 0.1]
        g = fem.gravity_direct(x, mesh.xyz, mesh.tet, model.rho, G)
        ratio = -np.einsum('ij,ij->i', g, x) / ((4.0 / 3.0) * np.pi * G * np.einsum('ij,ij->i', x, x))
        assert abs(ratio.mean() - 1.0) < 0.05
        errs.append(np.sqrt(np.mean((g + (4.0 / 3.0) * np.pi * G * x) ** 2)))
    assert errs[1] < errs[0]


# ------------------------------------------------------------ filter steps
def test_jackson_and_step_coeffs_vs_numpy_chebval():
    gam, c, e = filtlan.filter_coeffs(0.0, 10.0, 2.0, 4.0, 60)
    assert filtlan.jackson(60)[0] == pytest.approx(1.0)
    t = np.linspace(-1, 1, 101)
    assert np.allclose(filtlan.cheb_eval(gam, t), np.polynomial.chebyshev.chebval(t, gam), atol=1e-13)
    p = filtlan.cheb_eval(gam, (np.array([0.5, 3.0, 9.0]) - c) / e)
    assert p[1] > 0.9 and p[0] < 0.05 and p[2] < 0.05


def test_cheb_solve_converges_to_direct_solve_within_bound(ball):
    _, S, _, _, _, _ = ball
    rng = np.random.default_rng(0)
    W = rng.standard_normal((S.n, 3))
    exact = spla.spsolve(S.M.tocsc(), W)
    dinv = 1.0 / S.M.diagonal()
    lo, hi = filtlan.MASS_LO, filtlan.MASS_HI
    rate = (np.sqrt(hi / lo) - 1) / (np.sqrt(hi / lo) + 1)
    Mm = S.M
    for k in (10, 20, 40):
        X = filtlan.cheb_solve(Mm, dinv, W, k)
        E = X - exact
        # error in the M-norm bounded by 2 rate^k times the initial error
        e_now = np.sqrt(np.einsum('ij,ij->j', E, Mm @ E))
        e_0 = np.sqrt(np.einsum('ij,ij->j', exact, Mm @ exact))
        assert (e_now <= 2 * rate ** k * e_0 * (1 + 1e-9)).all()
    X = filtlan.cheb_solve(Mm, dinv, W, 80)
    assert np.abs(X - exact).max() <= 1e-12 * np.abs(exact).max()


def test_filter_apply_matches_spectral_evaluation(ball):
    """Recurrence == p((B - c)/e) Y evaluated through an eigendecomposition."""
    _, S, K, M, _, _ = ball
    op = filtlan.Operator(S, k_M=12)
    n = S.n
    PM = op.Minv(np.eye(n))
    B = PM @ K
    wB, VB = np.linalg.eig(B)
    gam, c, e = filtlan.filter_coeffs(-1.0, 5000.0, 0.0, 9.0, 30)
    Y = np.random.default_rng(1).standard_normal((n, 2))
    Z = filtlan.filter_apply(op, gam, c, e, Y)
    pw = filtlan.cheb_eval(gam, ((wB - c) / e).real)
    Zs = (VB @ (pw[:, None] * np.linalg.solve(VB, Y))).real
    assert np.abs(Z - Zs).max() <= 1e-9 * np.abs(Zs).max()


def test_lanczos_slice_matches_dense(ball):
    w, S, K, M, lam, _ = ball
    op = filtlan.Operator(S, k_M=40)
    lo, hi = filtlan.spectrum_bounds(op, S.n)
    assert hi >= lam[-1] and lo <= lam[0]
    lam_lo, lam_hi = -1e-8 * hi, 9.0
    got, X, res, info = filtlan.lanczos_slice(op, lam_lo, lam_hi, 100, 8, 16, bounds=(lo, hi))
    ref = lam[(lam >= lam_lo) & (lam <= lam_hi)]
    assert len(got) == len(ref) == 16
    big = np.abs(ref) > 1e-10 * lam[-1]
    assert np.allclose(got[big], ref[big], rtol=1e-10)
    assert np.abs(got[~big]).max() <= 1e-10 * lam[-1]
    assert res.max() <= 1e-6
    # cross-check the residual with the dense pencil
    r2 = eig.residuals(K, M, got, X, floor=filtlan.residual_floor(lam_lo, lam_hi))
    assert r2.max() <= 1e-6


def test_lanczos_empty_slice_stops_early(ball):
    """A slice inside a gap of the dense spectrum (no eigenvalue in [8, 10.5]
    on this mesh): every wanted Ritz value of p(B) belongs to an eigenvalue
    outside it, so once they have converged the run returns no pair before
    its block limit."""
    w, S, K, M, lam, _ = ball
    assert not ((lam >= 8.0) & (lam <= 10.5)).any()
    op = filtlan.Operator(S, k_M=30, k_P=30)
    got, X, res, info = filtlan.lanczos_slice(op, 8.0, 10.5, 200, 4, 16, seed=1)
    assert len(got) == 0 and info["blocks"] < 16


# ------------------------------------------------------------ rotation
def _ball_T2(h, omega):
    mesh, model = homogeneous_ball(h=h, seed=1)
    model.Omega = np.array([0.0, 0.0, omega])
    S = fem.assemble(mesh, model)
    w, X = eig.eigs_near(S, 2.55 ** 2, 16)
    o = np.argsort(w)
    w, X = w[o], X[:, o]
    sel = w > 1.0
    return S, w[sel], X[:, sel]


def test_coriolis_matrix_skew():
    mesh, model = layered_planet(h=0.25, seed=7, omega=0.3)
    S = fem.assemble(mesh, model)
    assert abs(S.R + S.R.T).max() <= 1e-15 * abs(S.R).max()
    x = np.random.default_rng(0).standard_normal(S.n)
    assert abs(x @ (S.R @ x)) <= 1e-12 * np.linalg.norm(x) ** 2 * abs(S.R).max()


def test_toroidal_coriolis_splitting():
    """First-order Coriolis splitting of a toroidal multiplet of a
    homogeneous ball: omega_m = omega_0 + m Omega / (l (l+1)), so the
    Hermitian matrix i X^T R X on the 0T2 eigenspace has eigenvalues
    m Omega / 6, m = -2..2 (basis independent)."""
    omega = 0.05
    errs = []
    for h in (0.45, 0.3):
        S, w, X = _ball_T2(h, omega)
        T2 = X[:, :5]
        ev = np.sort(np.linalg.eigvalsh(1j * (T2.T @ (S.R @ T2)))) * 6.0 / omega
        errs.append(np.abs(ev - np.arange(-2, 3)).max())
    assert errs[1] < errs[0] < 0.05 and errs[1] < 0.01


def test_rotating_reduction_identities():
    S, w, X = _ball_T2(0.45, 0.05)
    Xe, lam = X[:, :10], w[:10]
    # Omega = 0: omega_e = sqrt(Lambda_e) exactly (Sec. 7)
    wr0, _ = eig.rotating_reduced(lam, np.zeros((10, 10)))
    assert np.allclose(np.sort(wr0[wr0 > 0]), np.sqrt(lam), rtol=1e-13)
    # rotating: real spectrum in +- pairs
    Q = Xe.T @ (S.R @ Xe)
    wr, Y = eig.rotating_reduced(lam, Q)
    assert np.allclose(np.sort(wr), -np.sort(wr)[::-1], atol=1e-12)
    # orthogonality in the rotating inner product (eq. orthonormalcond):
    # b_H(u_i, u_j) - 2i (w_i + w_j)^{-1} c_r(u_i, u_j) = 0 for i != j
    pos = np.nonzero(wr > 0)[0]
    U = Xe @ Y[:10, pos]
    Mu = S.M @ U
    Ru = S.R @ U
    B = U.conj().T @ Mu
    Cr = U.conj().T @ Ru
    wi = wr[pos]
    G = B - 2j * Cr / (wi[:, None] + wi[None, :])
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-10 * np.abs(np.diag(G)).max()
    assert (np.diag(G).real > 0).all()


# ------------------------------------------------------------ gravity terms with a prescribed field
def _two_layer(h, rho_s, rho_f, kap_f=1.0, mu_s=1.0, lam_s=2.0, N2=0.0, r_core=0.5):
    """Solid core (radius r_core) inside a fluid shell, homogeneous layers."""
    m = layered_ball(radii=(r_core, 1.0), h=h, fluid_layers=(1,), seed=5)
    fl = m.region == 1
    nt = m.nt
    mdl = Model(rho=np.where(fl, rho_f, rho_s), lam=np.where(fl, kap_f, lam_s), mu=np.where(fl, 0.0, mu_s),
                N2=np.where(fl, N2, 0.0), G=0.0, Omega=np.zeros(3))
    return m, mdl


def _p2_nodes(m):
    dm = fem.dof_map(m.tet, m.region, m.nv)
    return dm, fem.p2_coords(m.xyz, dm.edges)


def test_core_buoyancy_closed_form():
    """Archimedes in a fixed linear field g' = -gamma x (Cowling, Sec. 2.3).

    Translating a homogeneous solid core rigidly by a inside a fluid of
    density rho_f costs, in the solid gravity volume terms,
    rho_s gamma V |a|^2 (from -rho u.(grad g').v; the two other terms vanish
    for a constant field), and in the fluid-solid interface term
    S{(v.g')(nu.u) rho_f}, by the divergence theorem over the core,
    rho_f int_core a.grad(a.g') = -rho_f gamma V |a|^2. With g' linear the
    P2 interpolants of the nodal products are exact, so
    a^T A_G a / a^T M a = gamma (1 - rho_f / rho_s) to rounding. A dropped
    interface term gives gamma, a flipped one gamma (1 + rho_f/rho_s), the
    solid density in place of the fluid one 0. Rigid rotations of the core
    cost nothing (u.g' = 0 and the two derivative terms cancel)."""
    gamma, rho_s, rho_f = 1.7, 2.6, 1.9
    m, mdl = _two_layer(0.3, rho_s, rho_f)
    dm, x = _p2_nodes(m)
    S = fem.assemble(m, mdl, gprime=-gamma * x)
    ns = int((dm.unode_solid >= 0).sum())
    xs = S.node_xyz[S.dm.u_p2[:ns]]
    for a in (np.array([1.0, 0.0, 0.0]), np.array([0.3, -0.8, 0.5])):
        u = np.zeros((S.dm.Nu, 3))
        u[:ns] = a
        u = u.ravel()
        ray = u @ (S.A_G @ u) / (u @ (S.M @ u))
        assert ray == pytest.approx(gamma * (1.0 - rho_f / rho_s), rel=1e-10)
    for axis in np.eye(3):
        u = np.zeros((S.dm.Nu, 3))
        u[:ns] = np.cross(axis, xs)
        u = u.ravel()
        assert abs(u @ (S.A_G @ u)) <= 1e-12 * abs(S.A_G).max() * (u @ u)


def test_fluid_buoyancy_matrix_for_a_constant_field():
    """With a constant field g' = c the fluid buoyancy term
    int rho N^2 (g'.v)(g'.u) / |g'|^2 is N^2 M_rho (x) c c^T / |c|^2 exactly
    (the direction enters, not the magnitude: |c| = 2.5 here). A fluid ball
    has no other A_G term."""
    c = np.array([1.5, -2.0, 0.0])
    N2 = 0.04
    m = layered_ball(radii=(1.0,), h=0.45, fluid_layers=(0,), seed=3)
    nt = m.nt
    mdl = Model(rho=np.full(nt, 1.3), lam=np.full(nt, 2.0), mu=np.zeros(nt), N2=np.full(nt, N2), G=0.0,
                Omega=np.zeros(3))
    dm, x = _p2_nodes(m)
    S = fem.assemble(m, mdl, gprime=np.tile(c, (len(x), 1)))
    ch = c / np.linalg.norm(c)
    ref = sps_kron(S.M_rho, N2 * np.outer(ch, ch))
    assert abs(S.A_G - ref).max() <= 1e-13 * abs(ref).max()


def sps_kron(A, B):
    import scipy.sparse as sps
    return sps.kron(A, sps.csr_matrix(B), format="csr")


def test_fluid_pressure_gravity_coupling_by_quadrature():
    """E_G in a fluid ball (eq. weakfluid2: int v.grad p - (v.g') p rho / kappa)
    against an independent Gauss rule on every tet: for a constant field c,
    a linear displacement u and a quadratic pressure q (all exact in P2),
    q^T E_G^T u = int u.grad q - (rho / kappa) (u.c) q. A dropped or flipped
    gravity part, or rho and kappa exchanged, moves it by O(1)."""
    rng = np.random.default_rng(4)
    c = np.array([0.7, -1.1, 0.4])
    rho, kap = 1.4, 2.3
    m = layered_ball(radii=(1.0,), h=0.45, fluid_layers=(0,), seed=3)
    nt = m.nt
    mdl = Model(rho=np.full(nt, rho), lam=np.full(nt, kap), mu=np.zeros(nt), N2=np.zeros(nt), G=0.0,
                Omega=np.zeros(3))
    dm, x = _p2_nodes(m)
    S = fem.assemble(m, mdl, gprime=np.tile(c, (len(x), 1)))
    A = rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    Qm = rng.standard_normal((3, 3))
    Qm = Qm + Qm.T
    qv = rng.standard_normal(3)
    ufun = lambda p: p @ A.T + b                       # linear vector field
    qfun = lambda p: np.einsum('ni,ij,nj->n', p, Qm, p) + p @ qv + 0.3
    dq = lambda p: 2.0 * p @ Qm + qv
    xu = S.node_xyz[S.dm.u_p2]
    xp = S.node_xyz[np.nonzero(S.dm.pnode >= 0)[0][np.argsort(S.dm.pnode[S.dm.pnode >= 0])]]
    lhs = qfun(xp) @ (S.E_G.T @ ufun(xu).ravel())
    pts, wts = _duffy_rule(4)
    total = 0.0
    for t in m.tet:
        v = m.xyz[t]
        J = (v[1:] - v[0]).T
        det = abs(np.linalg.det(J))
        p = v[0] + pts @ J.T
        uu = ufun(p)
        f = (uu * dq(p)).sum(1) - (rho / kap) * (uu @ c) * qfun(p)
        total += det * (wts @ f)
    assert lhs == pytest.approx(total, rel=1e-11)


# ------------------------------------------------------------ eigenvalue counts and the rotating reduction
def test_inertia_counts_pin_the_slice_count():
    """Sylvester's law: the number of eigenvalues of (K_eff, M) in
    [s1, s2) is the difference of the negative inertia of K_eff - s M at
    the two edges (LDL^T, another factorisation than the dense eigensolve)."""
    mesh, model = layered_planet(h=0.35, seed=7)
    S = fem.assemble(mesh, model)
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    for s1, s2 in ((16.0, 30.0), (30.0, 42.0)):
        # edges in gaps of the dense spectrum
        s1 = 0.5 * (lam[lam < s1].max() + lam[lam >= s1].min())
        s2 = 0.5 * (lam[lam < s2].max() + lam[lam >= s2].min())
        n_dense = int(((lam >= s1) & (lam < s2)).sum())
        assert n_dense > 0
        assert eig.inertia_count(K, M, s2) - eig.inertia_count(K, M, s1) == n_dense


def test_rotating_reduction_converges_to_full_problem():
    """The projected rotating problem (eq. sublinear0) on the m_e lowest
    eigenvectors approaches the full linearised quadratic problem (Sec. 7)
    as m_e grows, and equals it when the basis is complete. K is shifted by
    M (K + M is positive definite; both problems use the same shifted K)."""
    w = config_ball()
    model = w.model
    model.Omega = np.array([0.0, 0.0, 0.3])
    S = fem.assemble(w.mesh, model)
    K, M = eig.pencil_dense(S)
    K = K + M
    R = S.R.toarray()
    full = np.sort(eig.rotating_full(K, M, R))
    lam, X = eig.all_eigs(K, M)
    target = full[full > 0][:12]
    errs = []
    for me in (20, 60, 200, len(lam)):
        Xe = X[:, :me]
        wr, _ = eig.rotating_reduced(lam[:me], Xe.T @ R @ Xe)
        got = np.sort(wr[wr > 0])[:12]
        errs.append(np.abs(got / target - 1).max())
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] <= 1e-10

"""Pins of the self-gravitation oracle (Sec. 5.2, eqs. ph1body2,
ph1surface2, phi1fluidsolid, eigfull) against facts that do not come from
its own formulas: brute-force quadrature of the self distances, the charge
of a linear field, conservation of mass (the charges of any displacement
sum to zero), symmetry, the vanishing energy of a rigid translation of a
self-gravitating ball (which the Cowling operator alone does not give), and
toroidal modes that carry no mass and so do not move."""
import numpy as np
import pytest
from scipy import integrate

from oracle import eig, fem, p2, selfgrav
from synth.model import Model, homogeneous_ball, layered_planet


def _brute_tri(T, p):
    """int over the triangle of dS / |y - p| by adaptive quadrature (p off
    the plane)."""
    a, b, c = T
    area2 = np.linalg.norm(np.cross(b - a, c - a))
    f = lambda y, x: 1.0 / np.linalg.norm(a + x * (b - a) + y * (c - a) - p)
    return area2 * integrate.dblquad(f, 0, 1, 0, lambda x: 1 - x, epsabs=1e-13, epsrel=1e-12)[0]


def _duffy_tri_mean(T, p):
    """(1/|T|) int_T dS / |y - p| for p inside T: three sub-triangles with
    apex p in collapsed coordinates y = p + t (e0 + s (e1 - e0)), where the
    1/|y - p| singularity cancels against the Jacobian t |e0 x e1|, leaving
    |e0 x e1| int_0^1 ds / |e0 + s (e1 - e0)| (adaptive quadrature)."""
    total = 0.0
    for i in range(3):
        e0, e1 = T[i] - p, T[(i + 1) % 3] - p
        jac = np.linalg.norm(np.cross(e0, e1))
        total += jac * integrate.quad(lambda s: 1.0 / np.linalg.norm(e0 + s * (e1 - e0)), 0, 1,
                                      epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    area = 0.5 * np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0]))
    return total / area


def test_triangle_integral_matches_quadrature():
    rng = np.random.default_rng(11)
    for _ in range(6):
        T = rng.standard_normal((3, 3))
        p = rng.standard_normal(3)
        assert selfgrav._tri_inv_dist(T, p) == pytest.approx(_brute_tri(T, p), rel=1e-10)
    # a point almost in the plane, above an edge
    T = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    p = np.array([0.5, 0.0, 1e-3])
    assert selfgrav._tri_inv_dist(T, p) == pytest.approx(_brute_tri(T, p), rel=1e-8)


def test_face_self_distance_matches_duffy_quadrature():
    rng = np.random.default_rng(12)
    tris = rng.standard_normal((5, 3, 3))
    got = selfgrav.face_inv_R(tris)
    for T, v in zip(tris, got):
        assert v == pytest.approx(_duffy_tri_mean(T, T.mean(axis=0)), rel=1e-10)


def test_element_self_distance_by_cones_and_monte_carlo():
    # the cone identity int_K dx/|x - r| = sum_F (h_F / 2) int_F dS/|y - r|
    # with the face integrals by adaptive quadrature ...
    rng = np.random.default_rng(13)
    v = rng.standard_normal((4, 3))
    r = v.mean(axis=0)
    s = 0.0
    for f in ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)):
        T = v[list(f)]
        nrm = np.cross(T[1] - T[0], T[2] - T[0])
        s += 0.5 * abs(np.dot(r - T[0], nrm)) / np.linalg.norm(nrm) * _brute_tri(T, r)
    vol = abs(np.linalg.det(v[1:] - v[0])) / 6
    got = selfgrav.element_inv_R(v, np.array([[0, 1, 2, 3]]))[0]
    assert got == pytest.approx(s / vol, rel=1e-9)
    # ... and the mean of 1/|x - r| over uniform samples of the tet
    # (barycentric coordinates from sorted uniforms), 4 sigma
    u = np.sort(rng.random((400_000, 3)), axis=1)
    lam = np.diff(np.concatenate([np.zeros((len(u), 1)), u, np.ones((len(u), 1))], axis=1), axis=1)
    x = lam @ v
    vals = 1.0 / np.linalg.norm(x - r, axis=1)
    assert abs(vals.mean() - got) < 4 * vals.std() / np.sqrt(len(vals))


def _unit_ball(h=0.45, G=1.0 / np.pi):
    mesh, model = homogeneous_ball(h=h, seed=1)
    model.G = G
    return mesh, model


def test_charges_of_a_linear_field():
    """u = A x + c: an element carries rho tr(A) |K| and an outer face
    -rho |E| nu . u(barycentre) (the P2 interpolant is exact, and so is the
    edge-midpoint rule on a face for the linear integrand)."""
    mesh, model = _unit_ball()
    pts, inv_R, C = selfgrav.charges(mesh, model)
    dm = fem.dof_map(mesh.tet, mesh.region, len(mesh.xyz))
    X = fem.p2_coords(np.asarray(mesh.xyz), dm.edges)[dm.u_p2]
    rng = np.random.default_rng(14)
    A = rng.standard_normal((3, 3))
    c = rng.standard_normal(3)
    u = (X @ A.T + c).ravel()
    q = C @ u
    nt = mesh.nt
    vol, _ = p2.tet_geometry(np.asarray(mesh.xyz), np.asarray(mesh.tet))
    rho = np.asarray(model.rho)
    assert np.allclose(q[:nt], rho * np.trace(A) * vol, rtol=1e-12, atol=1e-14)
    ot, otri, oppv = selfgrav._outer_faces(mesh.tet)
    xyz = np.asarray(mesh.xyz)
    area, nrm = p2.face_geometry(xyz, otri)
    out = np.einsum('ij,ij->i', xyz[oppv] - xyz[otri[:, 0]], nrm) > 0
    nrm[out] *= -1.0
    bc = xyz[otri].mean(axis=1)
    expect = -rho[ot] * area * np.einsum('ij,ij->i', nrm, bc @ A.T + c)
    assert len(q) == nt + len(ot)
    assert np.allclose(q[nt:], expect, rtol=1e-12, atol=1e-14)
    assert np.allclose(pts[nt:], bc)


@pytest.mark.parametrize("constant_per_region", [True, False])
def test_total_charge_vanishes(constant_per_region):
    """Sum of all charges = int div(rho u) over the body, its surface parts
    included = 0 for any u (divergence theorem per element): with a density
    constant per region only the outer and fluid-solid faces carry surface
    charges; with the layered planet's per-element density every interior
    face across which it jumps does too."""
    mesh, model = layered_planet(h=0.25, seed=7)
    region = np.asarray(mesh.region)
    if constant_per_region:
        rho = np.where(region == fem.SOLID, 2.0, 0.7)
        model = Model(rho=rho, lam=model.lam, mu=model.mu, N2=model.N2, G=model.G, Omega=model.Omega)
    pts, inv_R, C = selfgrav.charges(mesh, model)
    n_fs = len(fem.fs_faces(mesh.tet, fem.dof_map(mesh.tet, region, len(mesh.xyz)).tet10, region, mesh.xyz)[0])
    n_out = len(selfgrav._outer_faces(mesh.tet)[0])
    n_jump = C.shape[0] - mesh.nt - n_out - n_fs
    assert n_fs > 0 and (n_jump == 0) == constant_per_region
    rng = np.random.default_rng(15)
    for _ in range(3):
        q = C @ rng.standard_normal(C.shape[1])
        assert abs(q.sum()) < 1e-12 * np.abs(q).sum()


def test_self_gravity_term_is_symmetric():
    """C^T S C is symmetric (S is: the point-mass kernel and its self terms).
    It is not definite: point masses at barycentres with the 1/R self term
    give a kernel matrix with some negative eigenvalues, unlike the
    continuous Newton kernel."""
    mesh, model = _unit_ball()
    pts, inv_R, C = selfgrav.charges(mesh, model)
    S = selfgrav.kernel_matrix(pts, inv_R, model.G)
    assert np.array_equal(S, S.T)
    T = selfgrav.self_gravity_dense(mesh, model)
    assert np.allclose(T, T.T, rtol=0, atol=1e-12 * np.abs(T).max())


def test_rigid_translation_energy_vanishes_under_refinement():
    """A rigid translation of a self-gravitating body changes no energy:
    its Rayleigh quotient under the full operator tends to 0 as h -> 0, while
    the Cowling operator gives about (4/3) pi G rho (the restoring force of
    the fixed reference field)."""
    rq = []
    for h in (0.45, 0.3):
        mesh, model = _unit_ball(h=h)
        sys = fem.assemble(mesh, model)
        K = fem.k_eff_dense(sys)
        M = sys.M
        pts, inv_R, C = selfgrav.charges(mesh, model)
        S = selfgrav.kernel_matrix(pts, inv_R, model.G)
        cow, full = [], []
        for c in range(3):
            u = np.zeros((sys.dm.Nu, 3))
            u[:, c] = 1.0
            u = u.ravel()
            m = u @ (M @ u)
            q = C @ u
            cow.append(u @ K @ u / m)
            full.append((u @ K @ u - q @ S @ q) / m)
        rq.append((np.array(cow), np.array(full)))
    four_thirds = 4.0 / 3.0 * np.pi * (1.0 / np.pi) * 1.0
    for cow, full in rq:
        assert np.all(np.abs(cow - four_thirds) < 0.1 * four_thirds)
        assert np.all(np.abs(full) < 0.05 * four_thirds)
    assert np.abs(rq[1][1]).max() < 0.25 * np.abs(rq[0][1]).max()


def test_toroidal_modes_carry_no_charge():
    """Toroidal motion of a homogeneous ball is divergence-free and tangent
    to the surface, so it carries no mass and self-gravitation leaves the
    0T2 multiplet where the Cowling operator puts it (the discrete charges
    vanish only in the limit: the gap shrinks under refinement), while the
    spheroidal 0S2 multiplet, which compresses the ball and moves its
    surface, drops by several percent."""
    gaps = []
    for h in (0.45, 0.3):
        mesh, model = _unit_ball(h=h)
        sys = fem.assemble(mesh, model)
        K = fem.k_eff_dense(sys)
        M = sys.M.toarray()
        T = selfgrav.self_gravity_dense(mesh, model)
        cow = eig.all_eigs(K, M)[0]
        full = eig.all_eigs(K - T, M)[0]
        # the six rigid modes, then 0T2 (5) and 0S2 (5)
        t2 = np.abs(np.sqrt(full[6:11]) / np.sqrt(cow[6:11]) - 1.0)
        s2 = np.sqrt(full[11:16]) / np.sqrt(cow[11:16]) - 1.0
        gaps.append(t2.max())
        assert t2.max() < 1e-4
        assert (s2 < -0.03).all()
    assert gaps[1] < gaps[0] / 3

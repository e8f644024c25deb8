"""Self-gravitation (NM_SELF_GRAVITY, Sec. 5.2 eq. eigfull) on the GPU
against the CPU oracle: the full operator K_eff - C^T S C applied to
blocks (FP64 and mixed), and slices of the full pencil of a homogeneous
self-gravitating ball (whose six rigid-body modes sit near zero) and of
the layered planet with a fluid core (fluid-solid faces charged) against
the dense oracle's eigenvalues.

Tolerances: the product adds one FP64 N-body sum (points ~ tets + faces,
summation order differs) and two sparse products to the K_eff product, so
the 1e-11 bound of K_eff holds; eigenvalues 1e-8 relative, 1e-10
lambda_max absolute for near-zero ones, residuals <= 1e-6."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.model import homogeneous_ball, layered_planet  # noqa: E402
from oracle import fem, eig, filtlan, selfgrav  # noqa: E402
from tests.helpers import to_internal, to_canonical, rel_err  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def nm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_11082_gb300 import nm as mod
    return mod


@pytest.fixture(scope="module")
def ctx(nm):
    return nm.Context(0)


def _ball():
    mesh, model = homogeneous_ball(h=0.45, seed=1)
    model.G = 1.0 / np.pi
    return mesh, model


@pytest.fixture(scope="module")
def sg_ball(nm, ctx):
    mesh, model = _ball()
    S = fem.assemble(mesh, model)
    T = selfgrav.self_gravity_dense(mesh, model)
    P = nm.Problem(ctx, mesh, model, self_gravity=True)
    return mesh, model, S, T, P


@pytest.fixture(scope="module")
def sg_planet(nm, ctx):
    mesh, model = layered_planet(h=0.25, seed=7)
    S = fem.assemble(mesh, model)
    T = selfgrav.self_gravity_dense(mesh, model)
    P = nm.Problem(ctx, mesh, model, self_gravity=True)
    return mesh, model, S, T, P


def test_charge_points_counted(sg_ball, sg_planet):
    for mesh, model, S, T, P in (sg_ball, sg_planet):
        assert P.info["n_charges"] == len(selfgrav.charges(mesh, model)[1]) > mesh.nt


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.mark.parametrize("which", ["ball", "planet"])
@pytest.mark.parametrize("b,ld", [(1, 1), (5, 7), (33, 33), (64, 70)])
def test_apply_full_operator_fp64(request, which, b, ld):
    mesh, model, S, T, P = request.getfixturevalue("sg_" + which)
    rng = np.random.default_rng(100 + b)
    Xc = rng.standard_normal((S.n, b))
    X = torch.zeros((S.n, ld), dtype=torch.float64, device=DEV)
    X[:, :b] = torch.tensor(to_internal(P, Xc), dtype=torch.float64, device=DEV)
    Y = torch.zeros_like(X)
    P.apply_K(X[:, :b], Y[:, :b], k_P=80)
    ref = filtlan.Operator(S, k_M=10, k_P=80).K(Xc) - T @ Xc
    assert rel_err(to_canonical(P, _host(Y[:, :b])), ref) <= 1e-11
    assert torch.count_nonzero(Y[:, b:]).item() == 0
    # the term itself is not negligible on these blocks
    assert np.linalg.norm(T @ Xc) > 1e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("b", [4, 32])
def test_apply_full_operator_mixed(nm, sg_planet, b):
    mesh, model, S, T, P = sg_planet
    Xc = np.random.default_rng(9).standard_normal((S.n, b))
    Y = torch.empty((S.n, b), dtype=torch.float64, device=DEV)
    P.apply_K(torch.tensor(to_internal(P, Xc), dtype=torch.float64, device=DEV), Y, k_P=28, prec=nm.NM_MIXED)
    ref = filtlan.Operator(S, k_M=28, k_P=28, refine=True).K(Xc) - T @ Xc
    assert rel_err(to_canonical(P, _host(Y)), ref) <= 1e-11


def test_float_products_are_unsupported(nm, sg_ball):
    mesh, model, S, T, P = sg_ball
    X = torch.zeros((S.n, 2), dtype=torch.float32, device=DEV)
    Y = torch.zeros_like(X)
    with pytest.raises(nm.NMError):
        P.apply_K(X, Y, k_P=10)


def _edges_in_gaps(lam, lo_idx, hi_idx):
    return 0.5 * (lam[lo_idx - 1] + lam[lo_idx]), 0.5 * (lam[hi_idx] + lam[hi_idx + 1])


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_slice_of_the_full_ball_pencil(nm, sg_ball, prec):
    """Slice [below the near-zero modes, a gap above the first seismic
    modes]: the six rigid-body modes of the full operator are near zero
    (the Cowling operator lifts the three translations to ~(4/3) pi G rho)."""
    mesh, model, S, T, P = sg_ball
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K - T, M)[0]
    assert np.abs(lam[:6]).max() < 0.1 and lam[6] > 1.0
    # upper edge in the widest gap among the 12th..30th eigenvalues
    k = 11 + int(np.argmax(np.diff(lam[11:31])))
    lo = lam[0] - 0.5
    hi = 0.5 * (lam[k] + lam[k + 1])
    P.set_interval(lo, hi, unit=nm.NM_UNIT_OMEGA2)
    p = nm.NM_F64 if prec == "f64" else nm.NM_MIXED
    res = P.lanczos_slice(block=8, degree=120, k_M=40, k_P=40, max_blocks=20, seed=5, prec=p)
    ref = lam[(lam >= lo) & (lam <= hi)]
    assert len(res.lam) == len(ref) == k + 1
    scale = 1e-10 * lam[-1]
    assert np.allclose(res.lam, ref, rtol=1e-8, atol=scale)
    assert res.resid.max() <= 1e-6
    res.free()


def _gapped_window(lam, lo, hi, sizes=range(8, 15)):
    """(i0, i1): a run of eigenvalues inside (lo, hi) whose edge gaps are
    the widest such pair (the slice edges sit in those gaps)."""
    best = None
    for i0 in np.nonzero((lam > lo) & (lam < hi))[0]:
        for cnt in sizes:
            i1 = i0 + cnt - 1
            if i0 < 1 or i1 + 1 >= len(lam):
                continue
            g = min(lam[i0] - lam[i0 - 1], lam[i1 + 1] - lam[i1])
            if best is None or g > best[0]:
                best = (g, i0, i1)
    return best[1], best[2]


def test_slice_of_the_full_planet_pencil(nm, sg_planet):
    """Fluid core: the fluid-solid faces carry rho_f nu . u^f - rho_s nu . u^s
    and the interior faces the per-element density jumps. The full operator
    of this coarse planet has ~370 negative and ~60 extra low modes below
    lambda ~ 8 that the Cowling operator does not have (element-average
    divergences of the fluid that K_eff leaves almost free, given negative
    energy by the point-mass self terms); above that the counts agree, so the
    slice sits in [10, 20]."""
    mesh, model, S, T, P = sg_planet
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K - T, M)[0]
    assert lam[0] < -1.0
    i0, i1 = _gapped_window(lam, 10.0, 20.0)
    lo, hi = _edges_in_gaps(lam, i0, i1)
    P.set_interval(lo, hi, unit=nm.NM_UNIT_OMEGA2)
    res = P.lanczos_slice(block=8, degree=600, k_M=20, k_P=20, max_blocks=40, check_every=2, prec=nm.NM_MIXED,
                          seed=2)
    ref = lam[(lam >= lo) & (lam <= hi)]
    assert len(res.lam) == len(ref) == i1 - i0 + 1
    assert np.allclose(res.lam, ref, rtol=1e-8, atol=1e-10 * lam[-1])
    assert res.resid.max() <= 1e-6
    res.free()

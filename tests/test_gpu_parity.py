"""GPU (libnm, through the C ABI) against the CPU oracle, element by element.

Sizes: the ~400-tet homogeneous ball and a coarse three-layer planet with a
fluid core and reference gravity, small enough for dense oracle solves yet
spanning many thread blocks, with ragged block widths (1, 5, 33, 64) and
leading dimensions larger than the width.

Tolerances (derived from the arithmetic): assembled FP64 values differ
only by summation order (atomics vs sorted COO): 1e-12 relative to the
largest entry. One FP64 SpMM / mass-solve / filter: 1e-12 .. 1e-9
relative (the filter runs d x k_M dependent steps). FP32 kernels: 2e-5
relative for one product (z ~ 30-60 terms of 6e-8 each), 1e-3 relative
for a whole FP32 filter application. Eigenvalues: 1e-8 relative (1e-10
lambda_max absolute for the rigid-body zero modes), residuals <= 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from synth.model import config_ball, layered_planet  # noqa: E402
from oracle import fem, eig, filtlan  # noqa: E402
from tests.helpers import gpu_csr_to_canonical, to_internal, to_canonical, rel_err  # noqa: E402

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


@pytest.fixture(scope="module")
def ball(nm, ctx):
    w = config_ball()
    S = fem.assemble(w.mesh, w.model)
    P = nm.Problem(ctx, w.mesh, w.model)
    return w, S, P


@pytest.fixture(scope="module")
def planet(nm, ctx):
    mesh, model = layered_planet(h=0.25, seed=7)
    S = fem.assemble(mesh, model)
    P = nm.Problem(ctx, mesh, model)
    return mesh, model, S, P


def _dev(a, dtype=torch.float64):
    return torch.tensor(a, dtype=dtype, device=DEV)


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


# ------------------------------------------------------------------ assembly
def test_ball_assembly_matches_oracle(ball):
    w, S, P = ball
    assert P.n == S.n and P.info["Np"] == 0
    AG = gpu_csr_to_canonical(P, 0)
    Mr = gpu_csr_to_canonical(P, 1)
    assert rel_err(AG.toarray(), S.A_G.toarray()) <= 1e-12
    assert rel_err(Mr.toarray(), S.M_rho.toarray()) <= 1e-12


def test_planet_assembly_matches_oracle(planet):
    mesh, model, S, P = planet
    assert P.n == S.n and P.Np == S.dm.Np and P.info["n_fs"] > 0
    canon, p2, _ = P.unodes()
    g = P.gravity()
    g_or = S.g_p2[p2]
    assert rel_err(g, g_or) <= 1e-12
    assert rel_err(gpu_csr_to_canonical(P, 0).toarray(), S.A_G.toarray()) <= 1e-12
    assert rel_err(gpu_csr_to_canonical(P, 1).toarray(), S.M_rho.toarray()) <= 1e-12
    assert rel_err(gpu_csr_to_canonical(P, 2).toarray(), (-S.A_p).toarray()) <= 1e-12
    assert rel_err(gpu_csr_to_canonical(P, 3).toarray(), S.E_G.toarray()) <= 1e-12
    assert rel_err(gpu_csr_to_canonical(P, 4).toarray(), S.E_G.T.toarray()) <= 1e-12


def test_supplied_gprime_is_used(nm, ctx, planet):
    mesh, model, S, _ = planet
    gp = S.g_p2 * 1.1
    P2 = nm.Problem(ctx, mesh, model, gprime=gp)
    _, p2, _ = P2.unodes()
    assert rel_err(P2.gravity(), gp[p2]) <= 1e-15


# ------------------------------------------------------------------ operator pieces
@pytest.mark.parametrize("b,ld", [(1, 1), (5, 7), (33, 33), (64, 70)])
def test_apply_K_M_R_match_oracle(planet, b, ld):
    mesh, model, S, P = planet
    rng = np.random.default_rng(b)
    Xc = rng.standard_normal((S.n, b))
    X = torch.zeros((S.n, ld), dtype=torch.float64, device=DEV)
    X[:, :b] = _dev(to_internal(P, Xc))
    Y = torch.zeros_like(X)
    op = filtlan.Operator(S, k_M=10, k_P=80)
    P.apply_K(X[:, :b], Y[:, :b], k_P=80)
    ref = op.K(Xc)
    assert rel_err(to_canonical(P, _host(Y[:, :b])), ref) <= 1e-11
    P.apply_M(X[:, :b], Y[:, :b])
    assert rel_err(to_canonical(P, _host(Y[:, :b])), S.M @ Xc) <= 1e-12
    # ld padding untouched
    assert torch.count_nonzero(Y[:, b:]).item() == 0


def test_apply_R_matches_oracle(nm, ctx):
    mesh, model = layered_planet(h=0.25, seed=7, omega=0.3)
    S = fem.assemble(mesh, model)
    P = nm.Problem(ctx, mesh, model)
    Xc = np.random.default_rng(0).standard_normal((S.n, 4))
    Y = torch.empty((S.n, 4), dtype=torch.float64, device=DEV)
    P.apply_R(_dev(to_internal(P, Xc)), Y)
    assert rel_err(to_canonical(P, _host(Y)), S.R @ Xc) <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 7, 40])
def test_solve_M_matches_oracle(planet, k):
    mesh, model, S, P = planet
    Wc = np.random.default_rng(k).standard_normal((S.n, 3))
    X = torch.empty((S.n, 3), dtype=torch.float64, device=DEV)
    P.solve_M(_dev(to_internal(P, Wc)), X, k_M=k)
    ref = filtlan.cheb_solve(S.M, 1.0 / S.M.diagonal(), Wc, k)
    assert rel_err(to_canonical(P, _host(X)), ref) <= 1e-12


def test_fp32_pieces(planet):
    mesh, model, S, P = planet
    Xc = np.random.default_rng(3).standard_normal((S.n, 8))
    X = _dev(to_internal(P, Xc), torch.float32)
    Y = torch.empty_like(X)
    P.apply_M(X, Y)
    assert rel_err(to_canonical(P, _host(Y)), S.M @ Xc) <= 2e-5
    P.apply_K(X, Y, k_P=40)
    op = filtlan.Operator(S, k_M=10, k_P=40)
    assert rel_err(to_canonical(P, _host(Y)), op.K(Xc)) <= 1e-4


# ------------------------------------------------------------------ filter
@pytest.mark.parametrize("which,d,kM,b", [("ball", 30, 12, 8), ("ball", 1, 2, 3), ("planet", 12, 8, 5)])
def test_filter_apply_fp64(ball, planet, nm, which, d, kM, b):
    S, P = (ball[1], ball[2]) if which == "ball" else (planet[2], planet[3])
    op = filtlan.Operator(S, k_M=kM, k_P=kM)
    lo, hi = filtlan.spectrum_bounds(op, S.n)
    gam, c, e = filtlan.filter_coeffs(lo, hi, 0.5, 9.0, d)
    Yc = np.random.default_rng(d).standard_normal((S.n, b))
    Z = torch.empty((S.n, b), dtype=torch.float64, device=DEV)
    P.filter_apply(gam, c, e, kM, _dev(to_internal(P, Yc)), Z, k_P=kM)
    ref = filtlan.filter_apply(op, gam, c, e, Yc)
    assert rel_err(to_canonical(P, _host(Z)), ref) <= 1e-9


def test_filter_apply_fp32(ball):
    _, S, P = ball
    op = filtlan.Operator(S, k_M=12)
    gam, c, e = filtlan.filter_coeffs(-1.0, 5000.0, 0.0, 9.0, 30)
    Yc = np.random.default_rng(0).standard_normal((S.n, 16))
    Z = torch.empty((S.n, 16), dtype=torch.float32, device=DEV)
    P.filter_apply(gam, c, e, 12, _dev(to_internal(P, Yc), torch.float32), Z)
    ref = filtlan.filter_apply(op, gam, c, e, Yc)
    assert rel_err(to_canonical(P, _host(Z)), ref) <= 1e-3


# ------------------------------------------------------------------ bounds and slices
def test_spectrum_bounds_enclose(ball):
    w, S, P = ball
    lo, hi = P.spectrum_bounds(steps=40, k_M=40)
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    assert lo <= lam[0] and hi >= lam[-1] and hi <= 1.2 * lam[-1]


def _check_slice(res, ref, lam_max):
    assert len(res.lam) == len(ref)
    big = np.abs(ref) > 1e-10 * lam_max
    assert np.allclose(res.lam[big], ref[big], rtol=1e-8)
    if (~big).any():
        assert np.abs(res.lam[~big]).max() <= 1e-10 * lam_max
    assert res.resid.max() <= 1e-6


def test_lanczos_slice_ball_fp64(ball):
    w, S, P = ball
    P.set_interval(0.0, 3.0)
    res = P.lanczos_slice(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5)
    K, M = eig.pencil_dense(S)
    lam, Xd = eig.all_eigs(K, M)
    ref = lam[(lam >= -1e-8 * lam[-1]) & (lam <= 9.0)]
    _check_slice(res, ref, lam[-1])
    # eigenspace: the computed vectors lie in the span of the reference ones
    X = to_canonical(P, _host(res.vectors()))
    sel = (lam >= -1e-8 * lam[-1]) & (lam <= 9.0)
    Q = Xd[:, sel]
    proj = X - Q @ (Q.T @ (M @ X))
    assert np.linalg.norm(proj) <= 1e-6 * np.linalg.norm(X)
    # M-orthonormal
    G = X.T @ (M @ X)
    assert np.abs(G - np.eye(len(res.lam))).max() <= 1e-8


def test_lanczos_slice_ball_fp32_filter(nm, ball):
    """A float filter leaves white rounding noise (~d x 6e-8) in the basis;
    the exact-pencil residual amplifies it by lambda_max / lambda, so only
    the eigenvalues (second order in the vector error) reach FP64 accuracy."""
    w, S, P = ball
    P.set_interval(0.0, 3.0)
    res = P.lanczos_slice(block=8, degree=100, k_M=28, k_P=28, max_blocks=16, seed=6, prec=nm.NM_F32,
                          tol=1e-2)
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    ref = lam[(lam >= -1e-8 * lam[-1]) & (lam <= 9.0)]
    assert len(res.lam) == len(ref)
    big = np.abs(ref) > 1e-10 * lam[-1]
    assert np.allclose(res.lam[big], ref[big], rtol=1e-6)
    assert res.resid.max() <= 1e-2


def test_lanczos_slice_ball_mixed(nm, ball):
    w, S, P = ball
    P.set_interval(0.0, 3.0)
    res = P.lanczos_slice(block=8, degree=100, k_M=28, k_P=28, max_blocks=16, seed=7, prec=nm.NM_MIXED)
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    ref = lam[(lam >= -1e-8 * lam[-1]) & (lam <= 9.0)]
    _check_slice(res, ref, lam[-1])


@pytest.mark.parametrize("k", [7, 28])
@pytest.mark.parametrize("b", [6, 32])
def test_solve_M_mixed_matches_refined_oracle(nm, planet, k, b):
    """b = 32 runs the lane-group float and double-float kernels with the
    fused first steps; b = 6 the generic ones."""
    mesh, model, S, P = planet
    Wc = np.random.default_rng(k).standard_normal((S.n, b))
    X = torch.empty((S.n, b), dtype=torch.float64, device=DEV)
    P.solve_M(_dev(to_internal(P, Wc)), X, k_M=k, prec=nm.NM_MIXED)
    ref = filtlan.refined_solve(S.M, 1.0 / S.M.diagonal(), Wc, k)
    # float semi-iterations add ~6e-8 x |residual| of noise
    tol = 1e-11 if k == 28 else 1e-8
    assert rel_err(to_canonical(P, _host(X)), ref) <= tol


@pytest.mark.parametrize("b,overlap", [(4, 0), (32, 0), (32, 1)])
def test_apply_K_mixed_matches_refined_oracle(nm, planet, b, overlap):
    """Also with the pressure chain on the problem's second stream
    (option overlap)."""
    mesh, model, S, P = planet
    Xc = np.random.default_rng(9).standard_normal((S.n, b))
    Y = torch.empty((S.n, b), dtype=torch.float64, device=DEV)
    try:
        P.set_option("overlap", overlap)
        P.apply_K(_dev(to_internal(P, Xc)), Y, k_P=28, prec=nm.NM_MIXED)
    finally:
        P.set_option("overlap", 0)
    op = filtlan.Operator(S, k_M=28, k_P=28, refine=True)
    assert rel_err(to_canonical(P, _host(Y)), op.K(Xc)) <= 1e-11


@pytest.mark.parametrize("b,ld", [(8, 8), (32, 32), (32, 40)])
def test_filter_apply_mixed(nm, planet, b, ld):
    """b = 32 runs the lane-group kernels, the fused first steps and the
    split carried by the combine; ld > b leaves the caller's blocks
    non-dense (the recurrence's own blocks stay dense)."""
    mesh, model, S, P = planet
    op = filtlan.Operator(S, k_M=20, k_P=20, refine=True)
    lo, hi = filtlan.spectrum_bounds(op, S.n)
    gam, c, e = filtlan.filter_coeffs(lo, hi, 0.5, 9.0, 20)
    Yc = np.random.default_rng(4).standard_normal((S.n, b))
    Ybuf = torch.zeros((S.n, ld), dtype=torch.float64, device=DEV)
    Ybuf[:, :b] = _dev(to_internal(P, Yc))
    Zbuf = torch.full((S.n, ld), 7.0, dtype=torch.float64, device=DEV)
    P.filter_apply(gam, c, e, 20, Ybuf[:, :b], Zbuf[:, :b], k_P=20, prec=nm.NM_MIXED)
    ref = filtlan.filter_apply(op, gam, c, e, Yc)
    assert rel_err(to_canonical(P, _host(Zbuf[:, :b])), ref) <= 1e-8
    if ld > b:
        assert bool((Zbuf[:, b:] == 7.0).all())     # padding columns untouched


@pytest.mark.parametrize("prec", ["f64", "mixed", "f32"])
def test_filter_degree_zero(nm, ball, prec):
    """A degree-0 filter is gamma_0 Y, exactly."""
    _, S, P = ball
    dt = torch.float32 if prec == "f32" else torch.float64
    Y = torch.randn((S.n, 5), dtype=dt, device=DEV)
    Z = torch.empty_like(Y)
    pr = {"f64": nm.NM_F64, "mixed": nm.NM_MIXED, "f32": nm.NM_F32}[prec]
    P.filter_apply(np.array([0.375]), 0.0, 1.0, 4, Y, Z, prec=pr)
    assert bool((Z == Y * 0.375).all())


def _planet_slice_edges(lam, lo_skip=4, count=12):
    """A slice of seismic modes well above the fluid band, edges in gaps."""
    hi_sel = lam[lam > 0.5]
    return 0.5 * (hi_sel[lo_skip - 1] + hi_sel[lo_skip]), 0.5 * (hi_sel[lo_skip + count - 1] + hi_sel[lo_skip + count])


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_lanczos_slice_planet(nm, planet, prec):
    """Fluid core: the filter must also suppress the fluid's essential
    spectrum near 0, so the degree follows the slice's distance from it."""
    mesh, model, S, P = planet
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    lo_edge, hi_edge = _planet_slice_edges(lam)
    P.set_interval(lo_edge, hi_edge, unit=1)
    res = P.lanczos_slice(block=8, degree=400, k_M=40 if prec == "f64" else 20, k_P=40 if prec == "f64" else 20,
                          max_blocks=30, seed=2, check_every=2,
                          prec=nm.NM_F64 if prec == "f64" else nm.NM_MIXED)
    ref = lam[(lam >= lo_edge) & (lam <= hi_edge)]
    _check_slice(res, ref, lam[-1])


def test_ritz_rotating_matches_oracle(nm, ctx):
    """Rotating reduction (eq. sublinear0) on the Ritz vectors of a slice:
    the eigenvalues depend only on the slice's eigenspace, so the GPU's
    (its own Lanczos vectors) and the oracle's (dense eigenvectors) agree."""
    from synth.model import homogeneous_ball
    mesh, model = homogeneous_ball(h=0.45, seed=1)
    model.Omega = np.array([0.0, 0.0, 0.05])
    S = fem.assemble(mesh, model)
    P = nm.Problem(ctx, mesh, model)
    P.set_interval(2.0, 3.0)
    res = P.lanczos_slice(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=3)
    K, M = eig.pencil_dense(S)
    lam, Xd = eig.all_eigs(K, M)
    sel = (lam >= 4.0) & (lam <= 9.0)
    assert len(res.lam) == sel.sum() == 10
    X = res.vectors()
    P.set_interval(2.0, 2.9)
    rot = P.ritz(X, mode=nm.NM_RITZ_ROTATING, lam_e=res.lam)
    Q = Xd[:, sel].T @ (S.R @ Xd[:, sel])
    wr, _ = eig.rotating_reduced(lam[sel], Q)
    ref = np.sort(wr[(wr >= 2.0) & (wr <= 2.9)])
    assert len(rot.lam) == len(ref) and len(ref) > 0
    assert np.allclose(np.sort(rot.lam), ref, rtol=1e-9)
    # the complex eigenvectors are returned; the full quadratic residual is
    # reported, not gated: with 10 basis modes and Omega = 0.05 the reduction's
    # truncation error is a few per cent
    U = rot.vectors()
    assert U.dtype == torch.complex128 and U.shape == (S.n, len(ref))
    assert np.isfinite(rot.resid).all() and rot.resid.max() < 0.1


def test_ritz_rotating_zero_omega(nm, ctx):
    """Omega = 0: omega_e = Lambda_e^{1/2} exactly (Sec. 7)."""
    from synth.model import homogeneous_ball
    mesh, model = homogeneous_ball(h=0.45, seed=1)
    P = nm.Problem(ctx, mesh, model)
    P.set_interval(2.0, 3.0)
    res = P.lanczos_slice(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=3)
    rot = P.ritz(res.vectors(), mode=nm.NM_RITZ_ROTATING, lam_e=res.lam)
    assert np.allclose(np.sort(rot.lam), np.sort(np.sqrt(res.lam)), rtol=1e-12)
    assert rot.resid.max() <= 1e-6


def test_empty_slice_reports_not_converged(nm, ball):
    w, S, P = ball
    P.set_interval(3.05, 3.1)   # gap between 0S2 and 1S1 on this mesh
    res = P.lanczos_slice(block=4, degree=40, k_M=20, k_P=20, max_blocks=3, seed=1, allow_unconverged=True)
    assert len(res.lam) == 0


def test_empty_slice_converges_early(nm, ball):
    """A slice in a gap of the dense spectrum ([8, 10.5] in lambda on this
    mesh) with a filter sharp enough to converge the eigenvalues around it:
    the run reports the slice converged with no pair before its block limit."""
    w, S, P = ball
    lam = eig.all_eigs(*eig.pencil_dense(S))[0]
    assert not ((lam >= 8.0) & (lam <= 10.5)).any()
    P.set_interval(8.0, 10.5, unit=nm.NM_UNIT_OMEGA2)
    res = P.lanczos_slice(block=4, degree=200, k_M=30, k_P=30, max_blocks=16, seed=1)
    assert len(res.lam) == 0 and res.info["blocks"] < 16
    res.free()


def test_invalid_block_width(nm, ball):
    _, S, P = ball
    X = torch.zeros((S.n, 65), dtype=torch.float64, device=DEV)
    with pytest.raises(nm.NMError) as e:
        P.apply_M(X, X.clone())
    assert e.value.code == nm.NM_EINVAL


@pytest.mark.parametrize("b", [8, 32])
def test_double_float_matches_double(nm, planet, b):
    """The mixed form's double-float SpMMs agree with the double ones to
    about 2^-48 per term; the float semi-iterations downstream then carry
    their own rounding (~6e-8 x the 1e-4-size refinement residual), so the
    outputs agree to ~1e-11 relative to the largest entry. b = 32 runs the
    lane-group (16-byte load) double-float kernels, b = 8 the generic ones."""
    mesh, model, S, P = planet
    Xc = np.random.default_rng(12).standard_normal((S.n, b))
    X = _dev(to_internal(P, Xc))
    Y0, Y1 = torch.empty_like(X), torch.empty_like(X)
    try:
        P.set_option("double_float", 0)
        P.apply_K(X, Y0, k_P=20, prec=nm.NM_MIXED)
        P.set_option("double_float", 1)
        P.apply_K(X, Y1, k_P=20, prec=nm.NM_MIXED)
        assert rel_err(_host(Y1), _host(Y0)) <= 2e-11
        P.set_option("double_float", 0)
        P.solve_M(X, Y0, 20, prec=nm.NM_MIXED)
        P.set_option("double_float", 1)
        P.solve_M(X, Y1, 20, prec=nm.NM_MIXED)
        assert rel_err(_host(Y1), _host(Y0)) <= 2e-11
    finally:
        P.set_option("double_float", 1)


def test_tile_options_agree(nm, planet):
    """Staged (both tiled variants, several tile heights) and unstaged float
    semi-iterations compute the same sums up to float rounding order."""
    mesh, model, S, P = planet
    W = _dev(np.random.default_rng(13).standard_normal((S.n, 32)), torch.float32)
    X = torch.empty_like(W)
    outs = []
    try:
        for tk, tr in ((1, 0), (1, 16), (2, 16), (2, 32), (2, 8)):
            P.set_option("tile_rows", tr)
            if tr:
                P.set_option("tile_kernel", tk)
            P.solve_M(W, X, 15)
            outs.append(_host(X))
    finally:
        P.set_option("tile_rows", 0)
        P.set_option("tile_kernel", 2)
    for o in outs[1:]:
        assert rel_err(o, outs[0]) <= 1e-5
    with pytest.raises(nm.NMError):
        P.set_option("tile_rows", 3)
    with pytest.raises(nm.NMError):
        P.set_option("no_such_option", 1)


@pytest.mark.parametrize("chunk", [256, 512, 1024])
def test_chunk_options_agree(nm, planet, chunk):
    """The chunked row schedule runs the same per-row code as the plain
    warp-per-row grid, so mass solves (float b = 32, double b = 40), the
    float pressure solve inside K_eff and a mixed filter agree with it to
    the last bits (bounded here by 1e-6 / 1e-14 relative)."""
    mesh, model, S, P = planet
    rng = np.random.default_rng(17)
    W32 = _dev(rng.standard_normal((S.n, 32)), torch.float32)
    W64 = _dev(rng.standard_normal((S.n, 40)))
    K64 = _dev(rng.standard_normal((S.n, 24)))
    lo, hi = P.spectrum_bounds(k_M=20)
    gam, c, e = nm.filter_design(lo, hi, 0.5, 9.0, 6)

    def run():
        X32, X64, Y32, Z = (torch.empty_like(W32), torch.empty_like(W64),
                            torch.empty_like(W32), torch.empty_like(K64))
        P.solve_M(W32, X32, 15)
        P.solve_M(W64, X64, 15)
        P.apply_K(W32, Y32, k_P=12)
        P.filter_apply(gam, c, e, 20, K64, Z, prec=nm.NM_MIXED)
        return [_host(v) for v in (X32, X64, Y32, Z)]

    try:
        P.set_option("vec", 0)          # the chunked schedule runs the scalar-gather row code
        base = run()
        P.set_option("chunk", chunk)
        got = run()
    finally:
        P.set_option("chunk", 0)
        P.set_option("vec", 1)
    for o, r, tol in zip(got, base, (1e-6, 1e-14, 1e-6, 1e-14)):
        assert rel_err(o, r) <= tol
    with pytest.raises(nm.NMError):
        P.set_option("chunk", 300)


def test_vec_option_agrees(nm, planet):
    """The 16-byte vectorised gathers (float, b = 32) sum each row in a
    different order than the scalar ones: float mass solve, float pressure
    solve inside K_eff and a whole FP32 filter agree with them to float
    rounding (1e-5 relative), and with the oracle as the FP32 tests state."""
    mesh, model, S, P = planet
    rng = np.random.default_rng(19)
    Wc = rng.standard_normal((S.n, 32))
    W32 = _dev(to_internal(P, Wc), torch.float32)
    op = filtlan.Operator(S, k_M=15, k_P=15)
    lo, hi = filtlan.spectrum_bounds(op, S.n)
    gam, c, e = filtlan.filter_coeffs(lo, hi, 0.5, 9.0, 8)

    def run():
        X, Y, Z = torch.empty_like(W32), torch.empty_like(W32), torch.empty_like(W32)
        P.solve_M(W32, X, 15)
        P.apply_K(W32, Y, k_P=15)
        P.filter_apply(gam, c, e, 15, W32, Z, k_P=15)
        return [_host(v) for v in (X, Y, Z)]

    vec = run()
    try:
        P.set_option("sched", 1)        # SM-local row order: same per-row code
        sched = run()
        P.set_option("sched", 0)
        P.set_option("vec", 0)
        scal = run()
    finally:
        P.set_option("vec", 1)
        P.set_option("sched", 0)
    for o, r in zip(sched, vec):
        assert rel_err(o, r) <= 1e-6
    for o, r in zip(vec, scal):
        assert rel_err(o, r) <= 1e-5
    assert rel_err(to_canonical(P, vec[1]), op.K(Wc)) <= 1e-4
    assert rel_err(to_canonical(P, vec[2]), filtlan.filter_apply(op, gam, c, e, Wc)) <= 1e-3
    with pytest.raises(nm.NMError):
        P.set_option("vec", 2)


@pytest.mark.parametrize("b", [8, 32])
def test_graph_replay_matches_eager(nm, planet, b):
    """Option graphs: degrees 1..d-1 of the mixed filter replayed from two
    captured CUDA graphs (gamma and the degree read on the device) give the
    eagerly launched result bit for bit."""
    mesh, model, S, P = planet
    lo, hi = P.spectrum_bounds(k_M=20)
    gam, c, e = nm.filter_design(lo, hi, 0.5, 9.0, 9)
    Y = _dev(np.random.default_rng(31).standard_normal((S.n, b)))
    Z0, Z1 = torch.empty_like(Y), torch.empty_like(Y)
    st = torch.cuda.Stream()           # capture needs a stream other than the legacy default
    with torch.cuda.stream(st):
        P.filter_apply(gam, c, e, 20, Y, Z0, prec=nm.NM_MIXED, stream=st)
        n0 = nm.kernel_launches()
        try:
            P.set_option("graphs", 1)
            P.filter_apply(gam, c, e, 20, Y, Z1, prec=nm.NM_MIXED, stream=st)
        finally:
            P.set_option("graphs", 0)
        n1 = nm.kernel_launches()
    st.synchronize()
    assert torch.equal(Z0, Z1)
    assert n1 - n0 > 9 * 40          # replayed kernels are counted


def test_graph_replay_batched_slices(nm, ball):
    """The batched recurrence (per-slice gamma table) under graph replay
    gives the eager eigenvalues exactly."""
    w, S, P = ball
    out = []
    for gflag in (0, 1):
        P.set_option("graphs", gflag)
        rs = P.lanczos_multi([(0.0, 2.7), (2.7, 3.0)], block=8, degree=100, k_M=20, k_P=20, max_blocks=16,
                             prec=nm.NM_MIXED, seed=4)
        out.append([r.lam.copy() for r in rs])
        for r in rs:
            r.free()
    P.set_option("graphs", 0)
    for a, b_ in zip(*out):
        assert np.array_equal(a, b_) and len(a) > 0


def test_autotune_report_and_results(nm, planet):
    """The autotuner times the kernel variants on the problem, keeps the
    fastest, and the results stay those of the oracle."""
    mesh, model, S, P = planet
    rep = P.autotune(b=8, prec=nm.NM_MIXED, k_M=20)
    assert {"variants", "chosen", "us_per_column_degree"} <= set(rep)
    assert len(rep["variants"]) >= 4 and all(v["ms_per_degree"] > 0 for v in rep["variants"])
    Wc = np.random.default_rng(21).standard_normal((S.n, 6))
    X = torch.empty((S.n, 6), dtype=torch.float64, device=DEV)
    P.solve_M(_dev(to_internal(P, Wc)), X, k_M=20, prec=nm.NM_MIXED)
    ref = filtlan.refined_solve(S.M, 1.0 / S.M.diagonal(), Wc, 20)
    assert rel_err(to_canonical(P, _host(X)), ref) <= 1e-9


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_lanczos_multi_matches_single_slices(nm, ball, prec):
    """Two slices batched through one filter recurrence give each slice's
    dense-oracle eigenpairs (the slices share bounds and Chebyshev map)."""
    w, S, P = ball
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    slices = [(0.0, 2.7), (2.7, 3.0)]
    res = P.lanczos_multi(slices, block=8, degree=100, k_M=40 if prec == "f64" else 20,
                          k_P=40 if prec == "f64" else 20, max_blocks=16, seed=4,
                          prec=nm.NM_F64 if prec == "f64" else nm.NM_MIXED)
    assert len(res) == 2
    for (lo, hi), r in zip(slices, res):
        l = -1e-8 * lam[-1] if lo == 0 else lo * lo
        ref = lam[(lam >= l) & (lam <= hi * hi)]
        _check_slice(r, ref, lam[-1])


def test_lanczos_multi_rejects_too_wide(nm, ball):
    w, S, P = ball
    with pytest.raises(nm.NMError) as e:
        P.lanczos_multi([(0.0, 1.0)], block=65)
    assert e.value.code == nm.NM_EINVAL


def test_lanczos_multi_more_than_64_columns(nm, ball):
    """Three slices of 32 columns (96 > 64) are filtered in groups of two
    and one per block step; each slice reaches the dense oracle's pairs."""
    w, S, P = ball
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    slices = [(0.0, 2.58), (2.58, 2.7), (2.7, 3.0)]
    res = P.lanczos_multi(slices, block=32, degree=100, k_M=40, k_P=40, max_blocks=8, seed=4)
    assert len(res) == 3
    for (lo, hi), r in zip(slices, res):
        l = -1e-8 * lam[-1] if lo == 0 else lo * lo
        _check_slice(r, lam[(lam >= l) & (lam <= hi * hi)], lam[-1])


# ------------------------------------------------------------------ resumable block Lanczos
def test_lanczos_steps_equal_slice_call(nm, ball):
    """begin / step until no slice is active / finish computes what
    nm_lanczos_slice computes (same kernels in the same order: identical
    eigenvalues), and the result matches the dense oracle."""
    w, S, P = ball
    P.set_interval(0.0, 3.0)
    kw = dict(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5, check_every=2)
    whole = P.lanczos_slice(**kw)
    run = P.lanczos_begin(None, **kw)
    steps = 0
    while True:
        st = run.info(0)
        assert st["blocks"] == steps and st["active"] == 1
        active = run.step()
        steps += 1
        if active == 0:
            break
        assert steps < 16
    st = run.info(0)
    assert st["converged"] == 1 and st["active"] == 0 and st["blocks"] == steps
    res = run.finish()[0]
    assert res.info["blocks"] == whole.info["blocks"] == steps
    assert np.array_equal(res.lam, whole.lam)
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    _check_slice(res, lam[(lam >= -1e-8 * lam[-1]) & (lam <= 9.0)], lam[-1])


def test_lanczos_steps_two_slices_and_early_finish(nm, ball):
    """Two slices in one run (mixed form) step to the dense oracle's
    eigenpairs; finishing a run early returns Rayleigh-Ritz pairs of the
    current basis with NM_ENOTCONV; a step after the end is a no-op."""
    w, S, P = ball
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    slices = [(0.0, 2.7), (2.7, 3.0)]
    run = P.lanczos_begin(slices, block=8, degree=100, k_M=20, k_P=20, max_blocks=16, seed=4,
                          prec=nm.NM_MIXED)
    while run.step() > 0:
        pass
    assert run.step() == 0
    res = run.finish()
    for (lo, hi), r in zip(slices, res):
        l = -1e-8 * lam[-1] if lo == 0 else lo * lo
        _check_slice(r, lam[(lam >= l) & (lam <= hi * hi)], lam[-1])
    P.set_interval(0.0, 3.0)
    early = P.lanczos_begin(None, block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5)
    early.step()
    with pytest.raises(nm.NMError) as e:
        early.finish()
    assert e.value.code == nm.NM_ENOTCONV
    early = P.lanczos_begin(None, block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5)
    early.step()
    part = early.finish(allow_unconverged=True)[0]
    assert part.info["blocks"] == 1 and part.info["m"] == 8
    # abandoning a run without finishing it releases it
    P.lanczos_begin(None, block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5).free()


def test_lanczos_begin_reuses_bounds(nm, ball):
    """The spectrum bounds depend on (steps, k_M, seed); a second run with
    the same triple reuses them (identical lam_lo, lam_hi), and an option
    change makes the next run compute them again."""
    w, S, P = ball
    P.set_interval(0.0, 3.0)
    kw = dict(block=8, degree=60, k_M=40, k_P=40, max_blocks=4, seed=9)
    r1 = P.lanczos_begin(None, **kw)
    r1.step()
    a = r1.finish(allow_unconverged=True)[0]
    r2 = P.lanczos_begin(None, **kw)
    r2.step()
    b = r2.finish(allow_unconverged=True)[0]
    assert a.info["lam_lo"] == b.info["lam_lo"] and a.info["lam_hi"] == b.info["lam_hi"]
    np.testing.assert_array_equal(a.lam, b.lam)
    P.set_option("vec", 1)
    r3 = P.lanczos_begin(None, **kw)
    r3.step()
    c = r3.finish(allow_unconverged=True)[0]
    assert c.info["lam_hi"] == pytest.approx(a.info["lam_hi"], rel=1e-10)


# ------------------------------------------------------------------ staged (shared-memory) float mass step
@pytest.mark.parametrize("k", [2, 3, 20])
def test_tma_mass_step_matches_vectorised_kernel(nm, planet, k):
    """The shared-memory staged mass-step kernel (option tma, b = 32 float)
    computes the same float semi-iteration as the lane-group kernel: the
    refined mixed solve agrees to float rounding of the sums (different
    order), and with the oracle's refined solve at 1e-9."""
    mesh, model, S, P = planet
    Wc = np.random.default_rng(31).standard_normal((S.n, 32))
    W = _dev(to_internal(P, Wc))
    out = {}
    for tma in (0, 1):
        P.set_option("tma", tma)
        X = torch.empty((S.n, 32), dtype=torch.float64, device=DEV)
        P.solve_M(W, X, k_M=k, prec=nm.NM_MIXED)
        out[tma] = _host(X)
    P.set_option("tma", 0)
    assert rel_err(out[1], out[0]) <= 2e-6
    ref = filtlan.refined_solve(S.M, 1.0 / S.M.diagonal(), Wc, k)
    assert rel_err(to_canonical(P, out[1]), ref) <= (1e-9 if k == 20 else 1e-5)


def test_tma_filter_matches_oracle_and_reports_no_timeout(nm, planet):
    """A whole mixed filter application on 32 columns with the staged
    kernel matches the oracle's refined filter, and a Lanczos step after it
    reads a clear time-out flag."""
    mesh, model, S, P = planet
    op = filtlan.Operator(S, k_M=20, k_P=20, refine=True)
    lo, hi = filtlan.spectrum_bounds(op, S.n, steps=30, seed=1)
    g, c, e = filtlan.filter_coeffs(lo, hi, 10.0, 40.0, 12)
    Yc = np.random.default_rng(32).standard_normal((S.n, 32))
    Z = torch.empty((S.n, 32), dtype=torch.float64, device=DEV)
    P.set_option("tma", 1)
    P.filter_apply(g, c, e, 20, _dev(to_internal(P, Yc)), Z, k_P=20, prec=nm.NM_MIXED)
    ref = filtlan.filter_apply(op, g, c, e, Yc)
    assert rel_err(to_canonical(P, _host(Z)), ref) <= 1e-8
    P.set_interval(3.0, 6.0)
    run = P.lanczos_begin(None, block=32, degree=20, k_M=20, k_P=20, max_blocks=3, seed=3, prec=nm.NM_MIXED)
    run.step()
    run.free()
    P.set_option("tma", 0)


def test_tma_mass_step_many_tiles_per_cta(nm, ctx):
    """On a mesh with ~20 tiles per CTA (every stage reused many times, the
    producer waiting on released stages) the staged kernel agrees with the
    lane-group kernel and with the oracle's refined solve."""
    mesh, model = layered_planet(h=0.1, seed=7)
    P = nm.Problem(ctx, mesh, model)
    S = fem.assemble(mesh, model)
    Wc = np.random.default_rng(33).standard_normal((S.n, 32))
    W = _dev(to_internal(P, Wc))
    out = {}
    for tma in (0, 1):
        P.set_option("tma", tma)
        X = torch.empty((S.n, 32), dtype=torch.float64, device=DEV)
        P.solve_M(W, X, k_M=20, prec=nm.NM_MIXED)
        out[tma] = _host(X)
    assert rel_err(out[1], out[0]) <= 2e-6
    ref = filtlan.refined_solve(S.M, 1.0 / S.M.diagonal(), Wc, 20)
    assert rel_err(to_canonical(P, out[1]), ref) <= 1e-9
    P.free()


# ------------------------------------------------------------------ dense products on the tensor cores
def _scaled(rng, rows, cols, spread=6.0):
    """Gaussian entries with row and column scales over 10^(+-spread/2)
    and a few exact zeros, negatives and tiny (subnormal-range) values."""
    A = rng.standard_normal((rows, cols))
    A *= 10.0 ** rng.uniform(-spread / 2, spread / 2, (rows, 1))
    A *= 10.0 ** rng.uniform(-1, 1, (1, cols))
    A[rng.random((rows, cols)) < 0.01] = 0.0
    A[rng.random((rows, cols)) < 0.001] *= 1e-300
    return A


def _chunk_bound(Xk, Yk):
    """2^-48 sum over 64-term chunks of the contraction of 64 max|X| max|Y|
    per output entry: the splitting keeps each entry to 2^-52 of its row's
    (column's) largest entry in the chunk and drops piece products below
    2^-51 of the product of the two largest. Xk: K x I, Yk: K x J."""
    K = Xk.shape[0]
    out = np.zeros((Xk.shape[1], Yk.shape[1]))
    for k0 in range(0, K, 64):
        mx = np.abs(Xk[k0:k0 + 64]).max(axis=0)
        my = np.abs(Yk[k0:k0 + 64]).max(axis=0)
        out += 64.0 * np.outer(mx, my)
    return 2.0 ** -48 * out + 1e-290


@pytest.mark.parametrize("I,J,K", [(1, 1, 1), (70, 21, 1000), (64, 16, 64), (130, 33, 200003), (5, 40, 129)])
def test_gemm_tn_fp64_accuracy(nm, ctx, I, J, K):
    """C = alpha X^T Y + beta C (the Gram-Schmidt and Ritz projection shape)
    against the FP64 product of numpy within the splitting's bound; identical
    on a second call (deterministic split sums)."""
    rng = np.random.default_rng(I * 7 + J * 13 + K)
    X, Y = _scaled(rng, K, I), _scaled(rng, K, J)
    C0 = rng.standard_normal((J, I))           # column-major I x J
    alpha, beta = -1.5, 0.25
    ref = alpha * (X.T @ Y) + beta * C0.T
    Ct = _dev(C0)
    ctx.gemm_tn(_dev(X), _dev(Y), Ct, alpha=alpha, beta=beta)
    got = _host(Ct).T
    err = np.abs(got - ref)
    bound = abs(alpha) * _chunk_bound(X, Y) + 2.0 ** -50 * np.abs(beta * C0.T)
    assert (err <= bound).all(), float((err / bound).max())
    # and much tighter than a float product would be
    assert err.max() <= 1e-12 * np.abs(ref).max()
    Ct2 = _dev(C0)
    ctx.gemm_tn(_dev(X), _dev(Y), Ct2, alpha=alpha, beta=beta)
    assert torch.equal(Ct, Ct2)


@pytest.mark.parametrize("I,J,K", [(1, 1, 1), (1000, 32, 576), (333, 7, 65), (64, 64, 64), (100003, 16, 96)])
def test_gemm_nn_fp64_accuracy(nm, ctx, I, J, K):
    """D = alpha X Y + beta D (the W - V C and X = V S shape) against numpy
    FP64 within the splitting's bound."""
    rng = np.random.default_rng(I + J * 3 + K * 5)
    X = _scaled(rng, I, K)
    Y = _scaled(rng, K, J)
    D0 = rng.standard_normal((I, J))
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
        ref = alpha * (X @ Y) + beta * D0
        Dt = _dev(D0)
        ctx.gemm_nn(_dev(X), _dev(np.ascontiguousarray(Y.T)), Dt, alpha=alpha, beta=beta)
        err = np.abs(_host(Dt) - ref)
        bound = _chunk_bound(X.T, Y) + 2.0 ** -50 * np.abs(beta * D0)
        assert (err <= bound).all(), float((err / bound).max())


def test_dense_tc_option_agrees_with_dgemm(nm, ball):
    """A slice solved with the tensor-core products and with cuBLAS DGEMM
    (option dense_tc) gives the same eigenvalues to 1e-12."""
    w, S, P = ball
    P.set_interval(0.0, 3.0)
    kw = dict(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5)
    a = P.lanczos_slice(**kw)
    P.set_option("dense_tc", 0)
    b = P.lanczos_slice(**kw)
    P.set_option("dense_tc", 1)
    assert len(a.lam) == len(b.lam) == 16
    lam_max = np.abs(a.lam).max()
    assert np.allclose(a.lam, b.lam, rtol=1e-12, atol=1e-12 * lam_max)


# ------------------------------------------------------------------ continuous batching
def test_slice_joining_a_running_batch(nm, ball):
    """A slice added to a batch after two block steps (its own block counter,
    the run's shared bounds and filter) reaches the dense oracle's
    eigenpairs, as does the slice that was running; each equals the same
    slice solved alone to 1e-10; taking a slice releases it while the other
    keeps stepping."""
    w, S, P = ball
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    kw = dict(block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5, check_every=1)
    run = P.lanczos_begin([(0.0, 2.7)], **kw)
    run.step()
    run.step()
    j = run.add(2.7, 3.0, seed=77)
    assert j == 1 and run.info(1)["blocks"] == 0 and run.info(0)["blocks"] == 2
    done = {}
    while len(done) < 2:
        active = run.step()
        for q in (0, 1):
            if q not in done and not run.info(q)["active"]:
                done[q] = run.take(q)
        if active == 0:
            break
    assert sorted(done) == [0, 1]
    assert run.finish() == []          # every slice was taken
    for q, (lo, hi) in ((0, (0.0, 2.7)), (1, (2.7, 3.0))):
        l = -1e-8 * lam[-1] if lo == 0 else lo * lo
        ref = lam[(lam >= l) & (lam <= hi * hi)]
        _check_slice(done[q], ref, lam[-1])
        P.set_interval(lo, hi)
        alone = P.lanczos_slice(**dict(kw, seed=5 if q == 0 else 77))
        big = np.abs(alone.lam) > 1e-10 * lam[-1]
        assert np.allclose(done[q].lam[big], alone.lam[big], rtol=1e-10)


def test_take_running_slice_returns_current_ritz_pairs(nm, ball):
    w, S, P = ball
    run = P.lanczos_begin([(0.0, 3.0)], block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5)
    run.step()
    with pytest.raises(nm.NMError) as e:
        run.take(0)
    assert e.value.code == nm.NM_ENOTCONV
    with pytest.raises(nm.NMError) as e:
        run.take(0)                     # already taken
    assert e.value.code == nm.NM_EINVAL
    run2 = P.lanczos_begin([(0.0, 3.0)], block=8, degree=100, k_M=40, k_P=40, max_blocks=16, seed=5)
    run2.step()
    r = run2.take(0, allow_unconverged=True)
    assert r.info["blocks"] == 1
    with pytest.raises(nm.NMError) as e:
        run2.add(1.0, 0.5)              # lo > hi
    assert e.value.code == nm.NM_EINVAL
    run2.free()


# ------------------------------------------------------------------ rotating layered planet (Sec. 7)
def test_rotating_planet_batched_mixed_matches_oracle(nm, ctx):
    """Rotating three-layer planet (fluid core, reference gravity,
    Omega = 0.06781 about z): two adjacent slices of the seismic spectrum
    solved in one batched mixed-precision run, their Ritz vectors projected
    onto the rotating problem (eq. sublinear0); the reduced frequencies match
    the oracle's reduction built from the dense eigenvectors of the same
    slices to 1e-8, and the frequencies come in +- pairs."""
    from synth.model import OMEGA_EARTH_NONDIM
    mesh, model = layered_planet(h=0.25, seed=7, omega=OMEGA_EARTH_NONDIM)
    S = fem.assemble(mesh, model)
    K, M = eig.pencil_dense(S)
    lam = eig.all_eigs(K, M)[0]
    hi = np.sqrt(lam[lam > 0.5])
    s1 = (0.5 * (hi[3] + hi[4]), 0.5 * (hi[13] + hi[14]))
    s2 = (s1[1], 0.5 * (hi[25] + hi[26]))
    P = nm.Problem(ctx, mesh, model)
    res = P.lanczos_multi([s1, s2], block=8, degree=400, k_M=20, k_P=20, max_blocks=30, seed=2, check_every=2,
                          prec=nm.NM_MIXED)
    Xs = [r.vectors() for r in res]
    lam_e = np.concatenate([r.lam for r in res])
    assert (np.concatenate([r.resid for r in res]) <= 1e-6).all()
    Xe = torch.cat(Xs, dim=1).contiguous()
    P.set_interval(s1[0], s2[1])
    rot = P.ritz(Xe, mode=nm.NM_RITZ_ROTATING, lam_e=lam_e)
    # oracle: the same slices' dense eigenpairs, reduced with R
    w_ref, X_ref = eig.slice_eigs(K, M, s1[0] ** 2, s2[1] ** 2)
    assert np.allclose(np.sort(lam_e), w_ref, rtol=1e-8)
    wr, _ = eig.rotating_reduced(w_ref, X_ref.T @ (S.R @ X_ref))
    wr = np.sort(wr[(wr >= s1[0]) & (wr <= s2[1])])
    assert len(rot.lam) == len(wr) > 0
    assert np.allclose(np.sort(rot.lam), wr, rtol=1e-8)
    full = np.sort(eig.rotating_reduced(w_ref, X_ref.T @ (S.R @ X_ref))[0])
    assert np.allclose(full, -full[::-1], atol=1e-12 * np.abs(full).max())
    assert (rot.resid >= 0).all() and np.isfinite(rot.resid).all()
    P.free()

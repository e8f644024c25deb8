"""CPU oracle: the steps of the polynomial-filtered Lanczos method.

Test infrastructure (CPU oracle). The paper applies a polynomial filter
with a Lanczos eigensolver to the pencil A u = w^2 M u and touches A, M
and M^{-1} only through matrix-vector products (Sec. 6.2); it defers the
filter and Lanczos details to its references. The readings used here,
where the paper leaves the choice open, are:

* Mass solve (M^{-1} "by matrix-vector multiplications"): k_M steps of
  Chebyshev semi-iteration preconditioned by D = diag(M) with fixed bounds
  [1/4, (19 + sqrt(249))/8] of D^{-1}M (the spectrum of the Jacobi-scaled
  P2 element mass matrix; Wathen's element bound). Three-term form

      x_1 = D^{-1} w / theta,
      x_{k+1} = x_{k-1} + om_{k+1} (x_k - x_{k-1} + D^{-1}(w - M x_k)/theta),
      om_1 = 2, om_{k+1} = 1 / (1 - om_k / (4 sigma^2)),

  theta = (b + a)/2, delta = (b - a)/2, sigma = theta / delta. The result
  is a fixed symmetric polynomial P_M ~ M^{-1}.
* Filter: Chebyshev expansion of the indicator of the mapped slice
  [alpha, beta] in [-1, 1] with Jackson damping,
      mu_0 = (acos(alpha) - acos(beta)) / pi,
      mu_k = 2 (sin(k acos(alpha)) - sin(k acos(beta))) / (k pi),
      g_k  = ((1 - k/(d+2)) sin(a_d) cos(k a_d) + cos(a_d) sin(k a_d)/(d+2))
             / sin(a_d),  a_d = pi / (d + 2),
  gamma_k = g_k mu_k, applied to B = P_M K (K = A_G plus, with a fluid,
  E_G P_P E_G^T where P_P ~ (-A_p)^{-1} by the same semi-iteration) by
      T_0 = Y, T_1 = (B Y - c Y)/e, T_{k+1} = 2 (B T_k - c T_k)/e - T_{k-1},
      Z = sum_k gamma_k T_k,   c, e = centre, half-width of [l_lo, l_hi].
* Lanczos: block Lanczos on p(B) in the M inner product with full
  two-pass classical Gram-Schmidt against the whole basis, Cholesky-QR of
  each new block, then Rayleigh-Ritz of the pencil on the basis.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

MASS_LO = 0.25
MASS_HI = (19.0 + np.sqrt(249.0)) / 8.0


# ---------------------------------------------------------------- mass solve
def cheb_solve(A, dinv, W, k, lo=MASS_LO, hi=MASS_HI):
    """k steps of Jacobi-preconditioned Chebyshev semi-iteration for A X = W.

    A: sparse SPD (n, n); dinv: (n,) inverse diagonal; W: (n, b).
    """
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    x_prev = np.zeros_like(W)
    x = dinv[:, None] * W / theta
    om = 2.0
    for _ in range(1, k):
        om = 1.0 / (1.0 - om / (4.0 * sigma * sigma))
        r = W - A @ x
        x_new = x_prev + om * (x - x_prev + dinv[:, None] * r / theta)
        x_prev, x = x, x_new
    return x


def refined_solve(A, dinv, W, k):
    """One step of iterative refinement around the k-step semi-iteration:
    x = P W, e = P (W - A x), result x + e (error operator (I - P A)^2)."""
    x = cheb_solve(A, dinv, W, k)
    return x + cheb_solve(A, dinv, W - A @ x, k)


class Operator:
    """B = P_M K_eff on dof blocks, with the pieces of the FP64 pencil.

    refine=True applies every inner solve as a refined solve (the inverse
    the mixed-precision form applies: float semi-iterations around one
    double residual, here written out in double).
    """

    def __init__(self, sys, k_M, k_P=None, refine=False):
        self.sys = sys
        self.k_M = k_M
        self.k_P = k_M if k_P is None else k_P
        self.refine = refine
        self.M = sys.M
        self.dinv_M = 1.0 / sys.M.diagonal()
        self.negAp = -sys.A_p if sys.has_fluid() else None
        self.dinv_P = 1.0 / self.negAp.diagonal() if sys.has_fluid() else None

    def K_exact(self, X):
        """K_eff X with A_p^{-1} by a sparse direct solve (Rayleigh-Ritz)."""
        Y = self.sys.A_G @ X
        if self.negAp is not None:
            if getattr(self, '_lu', None) is None:
                import scipy.sparse.linalg as spla
                self._lu = spla.splu(self.negAp.tocsc())
            Y = Y + self.sys.E_G @ self._lu.solve(np.asarray(self.sys.E_G.T @ X))
        return np.asarray(Y)

    def K(self, X):
        Y = self.sys.A_G @ X
        if self.negAp is not None:
            q = self.sys.E_G.T @ X
            solve = refined_solve if self.refine else cheb_solve
            s = solve(self.negAp, self.dinv_P, np.asarray(q), self.k_P)
            Y = Y + self.sys.E_G @ s
        return np.asarray(Y)

    def Minv(self, W):
        solve = refined_solve if self.refine else cheb_solve
        return solve(self.M, self.dinv_M, W, self.k_M)

    def B(self, X):
        return self.Minv(self.K(X))


# ---------------------------------------------------------------- filter
def jackson(d):
    a = np.pi / (d + 2)
    k = np.arange(d + 1)
    return ((1 - k / (d + 2)) * np.sin(a) * np.cos(k * a) + np.cos(a) * np.sin(k * a) / (d + 2)) / np.sin(a)


def step_coeffs(alpha, beta, d):
    alpha = float(np.clip(alpha, -1.0, 1.0))
    beta = float(np.clip(beta, -1.0, 1.0))
    ta, tb = np.arccos(alpha), np.arccos(beta)
    mu = np.empty(d + 1)
    mu[0] = (ta - tb) / np.pi
    k = np.arange(1, d + 1)
    mu[1:] = 2.0 * (np.sin(k * ta) - np.sin(k * tb)) / (k * np.pi)
    return mu


def filter_coeffs(lam_lo, lam_hi, xi, eta, d):
    """gamma_k, centre c, half-width e for slice [xi, eta] of [lam_lo, lam_hi]."""
    c = 0.5 * (lam_hi + lam_lo)
    e = 0.5 * (lam_hi - lam_lo)
    alpha = (xi - c) / e
    beta = (eta - c) / e
    return jackson(d) * step_coeffs(alpha, beta, d), c, e


def cheb_eval(gamma, t):
    """p(t) = sum gamma_k T_k(t) for scalar/array t in [-1, 1]."""
    t = np.asarray(t, float)
    T0 = np.ones_like(t)
    s = gamma[0] * T0
    if len(gamma) == 1:
        return s
    T1 = t.copy()
    s = s + gamma[1] * T1
    for k in range(2, len(gamma)):
        T0, T1 = T1, 2 * t * T1 - T0
        s = s + gamma[k] * T1
    return s


def filter_apply(op: Operator, gamma, c, e, Y):
    """Z = p((B - c)/e) Y by the three-term recurrence."""
    d = len(gamma) - 1
    T_prev = Y
    Z = gamma[0] * Y
    if d == 0:
        return Z
    T = (op.B(Y) - c * Y) / e
    Z = Z + gamma[1] * T
    for k in range(1, d):
        T_next = 2.0 * (op.B(T) - c * T) / e - T_prev
        Z = Z + gamma[k + 1] * T_next
        T_prev, T = T, T_next
    return Z


# ---------------------------------------------------------------- bounds
def lanczos_bounds(op: Operator, n, steps=40, seed=0):
    """Extreme Ritz values of B (M inner product) and the last residual norm."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 1))
    v /= np.sqrt(np.vdot(v, op.M @ v))
    V = [v]
    alpha, beta = [], []
    v_prev = np.zeros_like(v)
    b_prev = 0.0
    for j in range(steps):
        w = op.B(v)
        a = float(np.vdot(v, op.M @ w))
        w = w - a * v - b_prev * v_prev
        for u in V:                      # full reorthogonalisation
            w = w - float(np.vdot(u, op.M @ w)) * u
        b = np.sqrt(max(float(np.vdot(w, op.M @ w)), 0.0))
        alpha.append(a)
        beta.append(b)
        if b == 0.0:
            break
        v_prev, v, b_prev = v, w / b, b
        V.append(v)
    T = np.diag(alpha) + np.diag(beta[:-1], 1) + np.diag(beta[:-1], -1)
    th, S = np.linalg.eigh(T)
    res = np.abs(beta[-1] * S[-1, :])
    return th, res


def spectrum_bounds(op: Operator, n, steps=40, seed=0):
    """[l_lo, l_hi] for the Chebyshev map of B: 40-step Lanczos estimate.

    l_hi = 1.01 (theta_max + |residual|) encloses the top. l_lo = min(0,
    theta_min) - 1e-6 l_hi: the bottom Ritz value without its (large,
    unconverged) residual; an undershoot delta only lets T_d grow to
    cosh(d sqrt(2 delta / e)) ~ 1 for delta << e / d^2.
    """
    th, res = lanczos_bounds(op, n, steps, seed)
    hi = (th[-1] + res[-1]) * 1.01
    lo = min(0.0, th[0]) - 1e-6 * hi
    return lo, hi


# ---------------------------------------------------------------- Lanczos
def m_orth(op, W):
    """Cholesky-QR in the M inner product; returns (Q, R) with W = Q R."""
    G = W.T @ (op.M @ W)
    G = 0.5 * (G + G.T)
    R = np.linalg.cholesky(G).T
    return sla.solve_triangular(R, W.T, trans='T', lower=False).T, R


def residual_floor(lam_lo, lam_hi):
    """Denominator floor for relative residuals of (near-)zero eigenvalues.

    ||K x - l M x|| / (max(|l|, f) ||M x||) with f = 1e-3 max(|lo|, |hi|):
    a relative residual is undefined at l = 0 (rigid-body modes), so
    eigenvalues below f are measured against the slice's own scale.
    """
    return 1e-3 * max(abs(lam_lo), abs(lam_hi))


def rel_residuals(KX, MX, lam, floor):
    r = np.linalg.norm(KX - MX * lam[None, :], axis=0)
    den = np.linalg.norm(MX, axis=0) * np.maximum(np.abs(lam), floor)
    return r / den


def rayleigh_ritz(op: Operator, V, lam_lo, lam_hi, Sw=None):
    """Ritz pairs of the pencil (K_eff, M) on span(V) inside [lam_lo, lam_hi].

    Sw (m x nw, orthonormal columns): coefficients of the converged Ritz
    vectors of p(B) above the threshold. Then only the pairs whose
    coefficient vector lies at least half in span(Sw) are kept; the others
    are spurious Ritz values of the whole basis (mixtures of directions from
    both sides of the slice)."""
    KV = op.K_exact(V)
    MV = op.M @ V
    H = V.T @ KV
    G = V.T @ MV
    H = 0.5 * (H + H.T)
    G = 0.5 * (G + G.T)
    w, S = sla.eigh(H, G)
    sel = (w >= lam_lo) & (w <= lam_hi)
    if Sw is not None:
        frac = np.sum((Sw.T @ S) ** 2, axis=0) / np.sum(S ** 2, axis=0)
        sel &= frac >= 0.5
    X = V @ S[:, sel]
    lam = w[sel]
    res = rel_residuals(KV @ S[:, sel], MV @ S[:, sel], lam, residual_floor(lam_lo, lam_hi))
    return lam, X, res


def lanczos_slice(op: Operator, lam_lo, lam_hi, d, b, max_blocks, seed=0,
                  bounds=None, tol=1e-6, check_every=1, Y0=None):
    """Filtered block Lanczos for the eigenpairs with lambda in the slice.

    Returns (lam, X, resid, info). Stops when every Ritz value of p(B) above
    the filter threshold tau has converged and the pencil Rayleigh-Ritz on
    the basis finds the slice's pairs with residual <= tol, counting only
    the pairs that lie in the span of those converged Ritz vectors (the
    eigenpairs of the filtered Lanczos that Sec. 6.2 adopts come from the
    Ritz vectors of the filtered operator above the threshold).
    """
    n = op.M.shape[0]
    if bounds is None:
        bounds = spectrum_bounds(op, n, seed=seed + 1)
    blo, bhi = bounds
    gamma, c, e = filter_coeffs(blo, bhi, lam_lo, lam_hi, d)
    pa = cheb_eval(gamma, np.clip((lam_lo - c) / e, -1, 1))
    pb = cheb_eval(gamma, np.clip((lam_hi - c) / e, -1, 1))
    tau = 0.8 * min(pa, pb) if lam_lo > blo else 0.8 * pb
    Y = np.random.default_rng(seed).standard_normal((n, b)) if Y0 is None else Y0
    V, _ = m_orth(op, Y)
    basis = [V]
    Tcols = []
    info = dict(blocks=0, tau=tau, c=c, e=e, bounds=bounds)
    lam = X = res = None
    empty_checks = 0
    for j in range(max_blocks):
        Vj = basis[-1]
        W = filter_apply(op, gamma, c, e, Vj)
        Vall = np.concatenate(basis, axis=1)
        H = np.zeros((Vall.shape[1], b))
        for _ in range(2):                      # CGS2
            C = Vall.T @ (op.M @ W)
            W = W - Vall @ C
            H += C
        Tcols.append(H)
        Q, R = m_orth(op, W)
        info['blocks'] = j + 1
        m = Vall.shape[1]
        T = np.zeros((m, m))
        col = 0
        for Hc in Tcols:
            T[:Hc.shape[0], col:col + b] = Hc
            col += b
        T = 0.5 * (T + T.T)
        th, S = np.linalg.eigh(T)
        resid_est = np.linalg.norm(R @ S[-b:, :], axis=0)
        wanted = th >= tau
        conv = wanted & (resid_est <= 1e-8 * np.maximum(np.abs(th), 1.0))
        basis.append(Q)
        if (j + 1) % check_every == 0 and wanted.any() and conv.sum() == wanted.sum():
            lam, X, res = rayleigh_ritz(op, Vall, lam_lo, lam_hi, Sw=S[:, wanted])
            if len(lam) and np.all(res <= tol):
                info['m'] = m
                return lam, X, res, info
            # empty slice: all wanted Ritz values of p(B) converged (they
            # belong to eigenvalues outside the slice; one inside would have
            # p >= tau) and no pair in the slice, at two consecutive checks
            # from the fourth block on
            empty_checks = empty_checks + 1 if len(lam) == 0 else 0
            if empty_checks >= 2 and j + 1 >= 4:
                info['m'] = m
                return lam, X, res, info
        elif (j + 1) % check_every == 0:
            empty_checks = 0
    Vall = np.concatenate(basis[:-1], axis=1)
    lam, X, res = rayleigh_ritz(op, Vall, lam_lo, lam_hi)
    info['m'] = Vall.shape[1]
    return lam, X, res, info

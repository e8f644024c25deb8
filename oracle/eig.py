"""CPU oracle: eigenpairs of the discrete pencil by dense library solves.

Test infrastructure (CPU oracle). The filtered-Lanczos solver is a method
for reaching exactly the eigenpairs of the discrete symmetric-definite
pencil (paper eq. gep, Sec. 6.2)

    A u = w^2 M u,  A = A_G (solid) or A_G - E_G A_p^{-1} E_G^T (Cowling),

inside a slice [w_lo^2, w_hi^2]. Their plain definition is a dense
generalized symmetric eigensolve (LAPACK sygvd through SciPy), written out
here for problems small enough to hold densely.

For a rotating body the paper projects the quadratic problem onto m_e
Ritz vectors X_e (eq. sublinear0, Sec. 7):

    [[0, L], [L, 2i X^T R X]] [y; w y] = w [[L, 0], [0, I]] [y; w y],

with L = diag(lambda_e), solved densely; u = X_e y. The full linearised
problem (before projection, Sec. 7) is also given for tiny meshes.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import fem


def pencil_dense(sys: fem.System):
    return fem.k_eff_dense(sys), sys.M.toarray()


def slice_eigs(K, M, lam_lo, lam_hi):
    """All (lambda, X) of K x = lambda M x with lam_lo <= lambda <= lam_hi.

    X is M-orthonormal (X^T M X = I).
    """
    w, X = sla.eigh(K, M, subset_by_value=(lam_lo, lam_hi))
    return w, X


def all_eigs(K, M):
    return sla.eigh(K, M)


def residuals(K, M, lam, X, floor=0.0):
    """||K x - l M x|| / (max(|l|, floor) ||M x||) per column (2-norms)."""
    KX = K @ X
    MX = M @ X
    r = np.linalg.norm(KX - MX * lam[None, :], axis=0)
    return r / (np.linalg.norm(MX, axis=0) * np.maximum(np.abs(lam), floor))


def inertia_count(K, M, sigma):
    """Number of eigenvalues of (K, M) below sigma (Sylvester's law, LDL^T)."""
    _, D, _ = sla.ldl(K - sigma * M)
    ev = []
    i = 0
    n = D.shape[0]
    while i < n:
        if i + 1 < n and D[i + 1, i] != 0.0:
            ev.extend(np.linalg.eigvalsh(D[i:i + 2, i:i + 2]))
            i += 2
        else:
            ev.append(D[i, i])
            i += 1
    return int(np.sum(np.asarray(ev) < 0))


def rotating_reduced(lam_e, Q):
    """Eigenpairs of the projected rotating problem (eq. sublinear0).

    lam_e: (m,) positive Ritz values lambda = w_N^2; Q = X_e^T R X_e (real,
    skew). Solves the 2m x 2m Hermitian-definite pencil and returns
    (omega (2m,), Y (2m, 2m)) sorted ascending; y = Y[:m] gives u = X_e y.
    """
    m = len(lam_e)
    L = np.diag(lam_e).astype(complex)
    A = np.zeros((2 * m, 2 * m), complex)
    A[:m, m:] = L
    A[m:, :m] = L
    A[m:, m:] = 2j * Q
    B = np.zeros((2 * m, 2 * m), complex)
    B[:m, :m] = L
    B[m:, m:] = np.eye(m)
    A = 0.5 * (A + A.conj().T)
    w, Y = sla.eigh(A, B)
    return w, Y


def rotating_full(K, M, R):
    """All eigenvalues of the full linearised QEP (Sec. 7) for tiny n.

    w^2 M u - 2 i w R u - K u = 0, linearised as
    [[0, K], [K, 2iR]] z = w [[K, 0], [0, M]] z with z = [u; w u].
    K must be positive definite here (no zero modes).
    """
    n = K.shape[0]
    A = np.zeros((2 * n, 2 * n), complex)
    A[:n, n:] = K
    A[n:, :n] = K
    A[n:, n:] = 2j * R
    B = np.zeros((2 * n, 2 * n), complex)
    B[:n, :n] = K
    B[n:, n:] = M
    A = 0.5 * (A + A.conj().T)
    return sla.eigh(A, B, eigvals_only=True)


def eigs_near(sys, sigma, k):
    """k eigenpairs of (K_eff, M) nearest sigma by shift-invert (ARPACK).

    (K_eff - sigma M) u = f is solved through the sparse saddle-point form
    [[A_G - sigma M, E_G], [E_G^T, A_p]] [u; p] = [f; 0] (the pressure
    constraint of Sec. 2.2.2 kept explicit), so K_eff is never formed.
    """
    import scipy.sparse as sps
    import scipy.sparse.linalg as spla
    n = sys.n
    if sys.has_fluid():
        Z = sps.bmat([[sys.A_G - sigma * sys.M, sys.E_G], [sys.E_G.T, sys.A_p]], format='csc')
    else:
        Z = (sys.A_G - sigma * sys.M).tocsc()
    lu = spla.splu(Z)

    def solve(f):
        rhs = np.zeros(Z.shape[0])
        rhs[:n] = f
        return lu.solve(rhs)[:n]

    op = spla.LinearOperator((n, n), matvec=solve, dtype=float)
    w, X = spla.eigsh(sys.A_G if not sys.has_fluid() else spla.aslinearoperator(sys.A_G),
                      k=k, M=sys.M, sigma=sigma, OPinv=op, which='LM', tol=1e-12)
    o = np.argsort(w)
    return w[o], X[:, o]

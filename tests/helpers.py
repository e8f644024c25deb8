"""Shared test helpers: node-order maps between libnm and the oracle."""
import numpy as np
import scipy.sparse as sps


def gpu_csr_to_canonical(P, which):
    """Exported libnm matrix as a scipy CSR in the oracle's canonical dof order."""
    rp, col, val = P.export(which)
    canon, _, pcanon = P.unodes()
    nrows = len(rp) - 1
    rb, cb = {0: (3, 3), 1: (1, 1), 2: (1, 1), 3: (3, 1), 4: (1, 3)}[which]
    row_map = canon if which in (0, 1, 3) else pcanon
    col_map = canon if which in (0, 1, 4) else pcanon
    ncols = len(col_map)
    r = np.repeat(np.arange(nrows), np.diff(rp))
    R = (rb * row_map[r])[:, None, None] + np.arange(rb)[None, :, None] + 0 * np.arange(cb)[None, None, :]
    Cc = (cb * col_map[col])[:, None, None] + np.arange(cb)[None, None, :] + 0 * np.arange(rb)[None, :, None]
    V = val.reshape(-1, rb, cb)
    return sps.coo_matrix((V.ravel(), (R.ravel(), Cc.ravel())), shape=(rb * nrows, cb * ncols)).tocsr()


def to_internal(P, Xc):
    """Canonical (n x b) block -> libnm internal row order."""
    canon, _, _ = P.unodes()
    b = Xc.shape[1]
    return np.ascontiguousarray(Xc.reshape(-1, 3, b)[canon].reshape(-1, b))


def to_canonical(P, Xi):
    canon, _, _ = P.unodes()
    b = Xi.shape[1]
    out = np.empty_like(Xi.reshape(-1, 3, b))
    out[canon] = Xi.reshape(-1, 3, b)
    return out.reshape(-1, b)


def rel_err(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)

"""Algorithm 1 ("Apply a compressed HBS matrix to a vector") -- oracle side.

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the printed algorithm: its upward pass loops over every node of each level
l = L..1 (the printed inner loop names level L for every l), and its downward pass loops over
every node of each level l = 0..L (the printed pass names no node loop). The root carries no
u-hat. With one level only (L = 0) the factorization is A = D. The transpose A^* is applied by
the same passes with U and V swapped and D replaced by D^* (real field, * = transpose,
Section 2.1). Several columns are applied at once (q is N x c).
"""

import numpy as np

from .tree import children, level_nodes


def apply(F, X, trans=False):
    """u = A q (or A^* q with ``trans``) for the factorization F, column block X (N x c)."""
    X = np.asarray(X, dtype=np.float64)
    one_d = X.ndim == 1
    if one_d:
        X = X[:, None]
    if X.shape[0] != F.N:
        raise ValueError("X must have N rows")
    Ub, Vb = (F.V, F.U) if trans else (F.U, F.V)
    Db = {t: (d.T if trans else d) for t, d in F.D.items()}
    out = np.zeros_like(X)
    if F.L == 0:
        out[:] = Db[1] @ X
        return out[:, 0] if one_d else out

    def rows(t):
        return slice(F.offsets[t], F.offsets[t] + F.sizes[t])

    q_hat, u_hat = {}, {}
    for level in range(F.L, 0, -1):                      # upward pass
        for tau in level_nodes(level):
            if level == F.L:
                q_hat[tau] = Vb[tau].T @ X[rows(tau)]
            else:
                a, b = children(tau)
                q_hat[tau] = Vb[tau].T @ np.vstack([q_hat[a], q_hat[b]])
    for level in range(0, F.L + 1):                     # downward pass
        for tau in level_nodes(level):
            if level == F.L:
                out[rows(tau)] = Ub[tau] @ u_hat[tau] + Db[tau] @ X[rows(tau)]
                continue
            a, b = children(tau)
            stacked = Db[tau] @ np.vstack([q_hat[a], q_hat[b]])
            if level > 0:
                stacked = stacked + Ub[tau] @ u_hat[tau]
            ra = q_hat[a].shape[0]
            u_hat[a], u_hat[b] = stacked[:ra], stacked[ra:]
    return out[:, 0] if one_d else out


def dense(F):
    """Dense N x N operator of the factorization: Algorithm 1 applied to the identity."""
    return apply(F, np.eye(F.N))

"""Dense primitives of Section 2 -- oracle side.

Test infrastructure only (see ``oracle/__init__.py``).

* Section 2.2: full QR ``B = Q R`` (Q square orthogonal, R upper triangular), here by
  Householder reflectors written out one at a time.
* Section 2.4: ``col(B, k)`` = k orthonormal columns spanning the column space of B, from an
  unpivoted (truncated) QR; ``null(B, k)`` = the last k columns of the full Q of B^*.
  The remark closing Section 2.4 is why no pivoting is needed: the method only applies them
  to random matrices or products with random matrices.
* The Moore-Penrose pseudo-inverse used in Eqs. (d_tau_part_1), (d_tau_part_2) and the root
  step of Algorithm 2. The paper does not say how it is computed; it is unique, so the oracle
  takes numpy's SVD-based ``pinv`` with no singular-value cutoff.

Householder convention (one fixed choice, shared by reading with the GPU path but not by code):
for x = (alpha, x_2..x_m), sigma = ||x_2..m||: if sigma == 0 the reflector is the identity
(tau = 0, beta = alpha); otherwise beta = -sign(alpha) ||x||, v = (1, x_2..m / (alpha - beta)),
tau = (beta - alpha) / beta, and (I - tau v v^T) x = beta e_1  (Golub & Van Loan, Alg. 5.1.1,
with LAPACK's sign choice).
"""

import math

import numpy as np


def householder(x):
    """Reflector (v, tau, beta) with (I - tau v v^T) x = beta e_1 and v[0] = 1."""
    x = np.asarray(x, dtype=np.float64)
    alpha = float(x[0])
    sigma = math.sqrt(float(np.dot(x[1:], x[1:])))
    v = np.zeros_like(x)
    v[0] = 1.0
    if sigma == 0.0:
        return v, 0.0, alpha
    beta = -math.copysign(math.hypot(alpha, sigma), alpha)
    v[1:] = x[1:] / (alpha - beta)
    tau = (beta - alpha) / beta
    return v, tau, beta


def householder_qr(B):
    """Unpivoted Householder QR of B (m x n), Section 2.2.

    Returns (reflectors, R): reflectors[j] = (v_j, tau_j) acting on rows j..m-1, and R (m x n,
    upper triangular) with B = H_0 H_1 ... H_{k-1} R, k = min(m, n).
    """
    R = np.array(B, dtype=np.float64, copy=True)
    m, n = R.shape
    reflectors = []
    for j in range(min(m, n)):
        v, tau, beta = householder(R[j:, j])
        # apply H_j = I - tau v v^T to the trailing rows, column by column
        R[j:, j:] = R[j:, j:] - tau * np.outer(v, v @ R[j:, j:])
        R[j, j] = beta
        R[j + 1:, j] = 0.0
        reflectors.append((v, tau))
    return reflectors, R


def full_q(reflectors, m):
    """The m x m orthogonal factor Q = H_0 H_1 ... H_{k-1}, formed explicitly."""
    Q = np.eye(m)
    for j, (v, tau) in enumerate(reflectors):
        # Q <- Q H_j, with H_j acting on coordinates j..m-1
        Q[:, j:] = Q[:, j:] - tau * np.outer(Q[:, j:] @ v, v)
    return Q


def col(B, k):
    """``col(B, k)``, Section 2.4: first k columns of Q from the unpivoted QR of B."""
    B = np.asarray(B, dtype=np.float64)
    if k > B.shape[0]:
        raise ValueError("col: k exceeds the number of rows")
    reflectors, _ = householder_qr(B)
    return full_q(reflectors, B.shape[0])[:, :k]


def null(B, k):
    """``null(B, k)``, Section 2.4: last k columns of the full Q of B^* (so B @ result = 0)."""
    B = np.asarray(B, dtype=np.float64)
    Bt = B.T
    if k > Bt.shape[0] - min(Bt.shape):
        raise ValueError("null: nullspace dimension is smaller than k")
    reflectors, _ = householder_qr(Bt)
    return full_q(reflectors, Bt.shape[0])[:, -k:]


def pinv(B):
    """Moore-Penrose pseudo-inverse B^dagger (SVD, no cutoff)."""
    return np.linalg.pinv(np.asarray(B, dtype=np.float64), rcond=0.0)

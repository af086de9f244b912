"""Randomized samples Y = A Omega, Z = A^* Psi (Algorithm 2, first block) -- oracle side.

Test infrastructure only (see ``oracle/__init__.py``).

A is either a dense matrix (products by numpy matmul, a library primitive) or a black box: a
callable ``op(X, trans)`` returning A X or A^* X, the only access to A that Section 1 assumes.
"""

import numpy as np

from .philox import gaussian_test_matrices


def sample_dense(A, Omega, Psi):
    """(Y, Z) = (A Omega, A^T Psi) for a dense real A."""
    A = np.asarray(A, dtype=np.float64)
    return A @ Omega, A.T @ Psi


def sample_blackbox(op, Omega, Psi):
    """(Y, Z) from a black-box operator: s products with A and s with A^*."""
    return op(Omega, False), op(Psi, True)


def sample(A_or_op, N, s, seed):
    """Full first block of Algorithm 2: draw Omega, Psi (Philox streams 0/1) and sample."""
    Omega, Psi = gaussian_test_matrices(N, s, seed)
    if callable(A_or_op):
        Y, Z = sample_blackbox(A_or_op, Omega, Psi)
    else:
        Y, Z = sample_dense(A_or_op, Omega, Psi)
    return Omega, Psi, Y, Z

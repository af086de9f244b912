"""Pins for the oracle's dense primitives (Section 2): QR, col, null, pseudo-inverse."""

import numpy as np
import pytest
import scipy.linalg

from hbs_inputs import gaussian
from oracle.linalg import col, full_q, householder, householder_qr, null, pinv


def test_householder_maps_to_e1():
    for seed in range(5):
        x = gaussian(9, seed)
        v, tau, beta = householder(x)
        Hx = x - tau * v * (v @ x)
        assert abs(Hx[0] - beta) < 1e-14 * np.linalg.norm(x)
        assert np.abs(Hx[1:]).max() < 1e-14 * np.linalg.norm(x)
        assert abs(abs(beta) - np.linalg.norm(x)) < 1e-14 * np.linalg.norm(x)
        assert np.sign(beta) == -np.sign(x[0])          # LAPACK sign choice
    v, tau, beta = householder(np.array([-3.0, 0.0, 0.0]))
    assert tau == 0.0 and beta == -3.0                   # sigma == 0: identity reflector


@pytest.mark.parametrize("m,n", [(7, 4), (30, 16), (30, 30), (12, 20), (120, 64)])
def test_qr_matches_lapack(m, n):
    B = gaussian((m, n), m * 100 + n)
    refl, R = householder_qr(B)
    Q = full_q(refl, m)
    assert np.allclose(Q @ R, B, atol=1e-13)
    assert np.allclose(Q.T @ Q, np.eye(m), atol=1e-14)
    assert np.allclose(np.tril(R, -1), 0.0)
    # LAPACK (dgeqrf/dorgqr via numpy) uses the same reflector convention: same Q and R
    Ql, Rl = np.linalg.qr(B, mode="complete")
    k = min(m, n)
    assert np.allclose(Q[:, :k], Ql[:, :k], atol=1e-12)
    assert np.allclose(R, Rl, atol=1e-12)


@pytest.mark.parametrize("n,s,k", [(16, 30, 10), (20, 30, 10), (64, 120, 40), (5, 9, 4)])
def test_null(n, s, k):
    B = gaussian((n, s), n + s)
    P = null(B, k)
    assert P.shape == (s, k)
    assert np.abs(B @ P).max() <= 1e-13 * np.abs(B).max() * s
    assert np.allclose(P.T @ P, np.eye(k), atol=1e-14)
    # when the nullspace has dimension exactly k, the projector is the textbook one
    if s - n == k:
        Ns = scipy.linalg.null_space(B)
        assert np.allclose(P @ P.T, Ns @ Ns.T, atol=1e-12)
    # with a larger nullspace, P spans a subspace of it
    Ns = scipy.linalg.null_space(B)
    assert np.allclose(Ns @ (Ns.T @ P), P, atol=1e-12)


def test_null_is_last_columns_of_full_q():
    B = gaussian((6, 14), 3)
    Ql, _ = np.linalg.qr(B.T, mode="complete")
    assert np.allclose(null(B, 5), Ql[:, -5:], atol=1e-13)


@pytest.mark.parametrize("n,k", [(16, 10), (80, 40), (10, 10)])
def test_col(n, k):
    B = gaussian((n, k), n * k)
    U = col(B, k)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-14)
    assert np.allclose(U @ (U.T @ B), B, atol=1e-12)
    Ql, _ = np.linalg.qr(B)
    assert np.allclose(U, Ql, atol=1e-12)               # same convention as LAPACK


def test_col_of_rank_deficient_product():
    # exact rank-k sample: col recovers the range (Section 2.3 randomized range finder)
    n, k = 40, 6
    W = gaussian((n, k), 1) @ gaussian((k, 60), 2)
    U = col(W @ gaussian((60, k), 3), k)
    assert np.linalg.norm(W - U @ (U.T @ W)) < 1e-12 * np.linalg.norm(W)


@pytest.mark.parametrize("n,s", [(16, 30), (80, 120), (30, 30)])
def test_pinv_penrose(n, s):
    B = gaussian((n, s), n + 7 * s)
    X = pinv(B)
    assert np.allclose(B @ X, np.eye(n), atol=1e-12)         # full row rank: B B^+ = I
    assert np.allclose(X @ B @ X, X, atol=1e-12)
    assert np.allclose((X @ B).T, X @ B, atol=1e-12)
    Xl = np.linalg.lstsq(B, np.eye(n), rcond=None)[0]         # minimum-norm solution
    assert np.allclose(X, Xl, atol=1e-12)

"""Pins for the oracle's Algorithm 2 (compression), Algorithm 1 (apply), sampling and norms.

Each pin ties the oracle to something other than itself: exact recovery of an exactly
HBS matrix assembled block by block (Section 3.2), the canonical-form identity of
Eq. (define_d_tau), the sample identity of Eq. (newtestmatrix), the root identity
D^(0) = A~^(1) (Section 3.3), the single-node special case (a least-squares solve), brute-force
products, and the textbook 2-norm. The last group plants plausible mistakes in the oracle and
checks that a pin catches each one.
"""

import numpy as np
import pytest

import oracle.compress as oc
from hbs_inputs import exact_hbs, gaussian
from oracle import apply as oa
from oracle.compress import HBSFactors, check_shape, compress
from oracle.norms import power_norm, relative_error
from oracle.philox import gaussian_test_matrices as draw_test_matrices
from oracle.sample import sample, sample_dense

_GOOD_MERGE = oc.merge

# (N, k, r, s, leaf_max): exact block rank k, r = k + p random vectors, s >= max(leaf + r, 3r)
OVERSAMPLED = [(400, 5, 8, 24, 16), (1000, 6, 9, 27, 18), (256, 4, 6, 18, 12), (97, 3, 5, 15, 10)]


def _case(N, k, r, s, leaf, seed=1):
    g = exact_hbs(N, leaf, k, seed)
    A = g.dense()
    Om, Ps = draw_test_matrices(N, s, seed + 10)
    return g, A, Om, Ps, A @ Om, A.T @ Ps


def _rel(X, Y):
    return np.linalg.norm(X - Y) / np.linalg.norm(Y)


def _recovery_error(N, k, r, s, leaf, seed=1):
    g, A, Om, Ps, Y, Z = _case(N, k, r, s, leaf, seed)
    F = compress(Om, Ps, Y, Z, r, leaf)
    return _rel(oa.dense(F), A)


@pytest.mark.parametrize("case", OVERSAMPLED)
def test_exact_recovery_oversampled(case):
    assert _recovery_error(*case) < 1e-11


def test_exact_recovery_without_oversampling():
    # r = k, s = 3k, leaf 16 (exact-HBS, N = 1024, k = 10): recovery holds, but with p = 0 the
    # sweep amplifies rounding (measured ~4e-9), so only a loose bound is a pin here.
    assert _recovery_error(1024, 10, 10, 30, 16) < 1e-7


def test_single_node_tree_is_least_squares():
    # L = 0: the root is the only node and D = Y Omega^dagger = A when N <= s
    N, s = 20, 26
    A = gaussian((N, N), 4)
    Om, Ps = draw_test_matrices(N, s, 5)
    F = compress(Om, Ps, A @ Om, A.T @ Ps, 3, 32)
    assert F.L == 0
    assert np.allclose(F.D[1], A, atol=1e-12)
    assert np.allclose(F.D[1], np.linalg.lstsq(Om.T, (A @ Om).T, rcond=None)[0].T, atol=1e-12)


def test_factor_invariants():
    N, k, r, s, leaf = OVERSAMPLED[0]
    g, A, Om, Ps, Y, Z = _case(N, k, r, s, leaf)
    F, blk = compress(Om, Ps, Y, Z, r, leaf, keep_blocks=True)
    for t in F.U:
        U, V, D = F.U[t], F.V[t], F.D[t]
        assert np.allclose(U.T @ U, np.eye(r), atol=1e-13)
        assert np.allclose(V.T @ V, np.eye(r), atol=1e-13)
        # canonical form: U^* D V = 0 follows from Eq. (d_tau_formula) for any input
        assert np.abs(U.T @ D @ V).max() < 1e-12 * max(1.0, np.abs(D).max())
        # Omega_tau P_tau = 0 for P = null(Omega_tau, r)
        P = oc.null(blk["Omega"][t], r)
        assert np.abs(blk["Omega"][t] @ P).max() < 1e-12 * np.abs(blk["Omega"][t]).max()


def test_leaf_discrepancy_matches_definition():
    # Eq. (define_d_tau): D_tau = A_tt - U U^* A_tt V V^* at the leaves, from dense A
    N, k, r, s, leaf = OVERSAMPLED[1]
    g, A, Om, Ps, Y, Z = _case(N, k, r, s, leaf)
    F = compress(Om, Ps, Y, Z, r, leaf)
    for t in range(2 ** F.L, 2 ** (F.L + 1)):
        o, n = F.offsets[t], F.sizes[t]
        Att = A[o:o + n, o:o + n]
        U, V = F.U[t], F.V[t]
        assert np.allclose(F.D[t], Att - U @ U.T @ Att @ V @ V.T, atol=1e-11)


def _blockdiag(blocks):
    rows = sum(b.shape[0] for b in blocks)
    cols = sum(b.shape[1] for b in blocks)
    out = np.zeros((rows, cols))
    i = j = 0
    for b in blocks:
        out[i:i + b.shape[0], j:j + b.shape[1]] = b
        i, j = i + b.shape[0], j + b.shape[1]
    return out


def test_parent_samples_match_newtestmatrix_identity():
    # Eq. (newtestmatrix): (U^(L))^* (Y - D^(L) Omega) = A~^(L) (V^(L))^* Omega with
    # A~^(L) = (U^(L))^* A V^(L) (Eq. newdef1) formed densely
    N, k, r, s, leaf = OVERSAMPLED[0]
    g, A, Om, Ps, Y, Z = _case(N, k, r, s, leaf)
    F, blk = compress(Om, Ps, Y, Z, r, leaf, keep_blocks=True)
    leaves = range(2 ** F.L, 2 ** (F.L + 1))
    UL = _blockdiag([F.U[t] for t in leaves])
    VL = _blockdiag([F.V[t] for t in leaves])
    At = UL.T @ A @ VL
    lhs_Y = At @ VL.T @ Om                                   # rows: r per leaf, in leaf order
    lhs_Z = At.T @ UL.T @ Ps
    for i, t in enumerate(range(2 ** (F.L - 1), 2 ** F.L)):  # parents of the leaves
        assert np.allclose(blk["Y"][t], lhs_Y[2 * r * i:2 * r * (i + 1)], atol=1e-10)
        assert np.allclose(blk["Z"][t], lhs_Z[2 * r * i:2 * r * (i + 1)], atol=1e-10)
        assert np.allclose(blk["Omega"][t], (VL.T @ Om)[2 * r * i:2 * r * (i + 1)], atol=1e-12)


def test_root_block_is_coarsest_projection():
    # Section 3.3: D^(0) = A~^(1) = (Ubar^(1))^* A Vbar^(1) with expanded level-1 bases
    N, k, r, s, leaf = OVERSAMPLED[0]
    g, A, Om, Ps, Y, Z = _case(N, k, r, s, leaf)
    F = compress(Om, Ps, Y, Z, r, leaf)
    Ubar, Vbar = {}, {}
    for level in range(F.L, 0, -1):
        for t in range(2 ** level, 2 ** (level + 1)):
            if level == F.L:
                Ubar[t], Vbar[t] = F.U[t], F.V[t]
            else:
                Ubar[t] = _blockdiag([Ubar[2 * t], Ubar[2 * t + 1]]) @ F.U[t]
                Vbar[t] = _blockdiag([Vbar[2 * t], Vbar[2 * t + 1]]) @ F.V[t]
    U1 = _blockdiag([Ubar[2], Ubar[3]])
    V1 = _blockdiag([Vbar[2], Vbar[3]])
    assert np.allclose(F.D[1], U1.T @ A @ V1, atol=1e-10)


def _generator_factors(g):
    return HBSFactors(N=g.N, r=g.k, L=g.L, offsets=g.offsets, sizes=g.sizes,
                      U=dict(g.U), V=dict(g.V), D=dict(g.D))


@pytest.mark.parametrize("N,leaf,k", [(400, 16, 5), (97, 10, 3), (64, 8, 4), (20, 32, 3)])
def test_apply_matches_blockwise_assembly(N, leaf, k):
    # Algorithm 1 on the generator's telescoping factors reproduces the matrix assembled
    # block by block from expanded bases (Section 3.2), for A and A^*
    g = exact_hbs(N, leaf, k, 3)
    A = g.dense()
    F = _generator_factors(g)
    X = gaussian((N, 5), 9)
    assert np.allclose(oa.apply(F, X), A @ X, atol=1e-12)
    assert np.allclose(oa.apply(F, X, trans=True), A.T @ X, atol=1e-12)
    assert np.allclose(oa.apply(F, X[:, 0]), A @ X[:, 0], atol=1e-12)


def test_sample_brute_force_integers():
    # integer-valued inputs: every product and sum is exact, compare with Python integers
    rng = np.random.default_rng(0)
    A = rng.integers(-5, 6, (9, 9)).astype(float)
    Om = rng.integers(-5, 6, (9, 4)).astype(float)
    Ps = rng.integers(-5, 6, (9, 4)).astype(float)
    Y, Z = sample_dense(A, Om, Ps)
    for i in range(9):
        for c in range(4):
            assert Y[i, c] == sum(int(A[i, j]) * int(Om[j, c]) for j in range(9))
            assert Z[i, c] == sum(int(A[j, i]) * int(Ps[j, c]) for j in range(9))


def test_sample_blackbox_equals_dense():
    g = exact_hbs(64, 8, 4, 5)
    A = g.dense()
    F = _generator_factors(g)
    _, _, Y1, Z1 = sample(A, 64, 12, 3)
    _, _, Y2, Z2 = sample(lambda X, t: oa.apply(F, X, t), 64, 12, 3)
    assert np.allclose(Y1, Y2, atol=1e-12) and np.allclose(Z1, Z2, atol=1e-12)


def test_power_norm_matches_two_norm():
    Q1, _ = np.linalg.qr(gaussian((60, 60), 1))
    Q2, _ = np.linalg.qr(gaussian((60, 60), 2))
    sv = np.concatenate([[10.0], np.linspace(1.0, 0.1, 59)])
    B = Q1 @ np.diag(sv) @ Q2.T
    est = power_norm(lambda x: B @ x, lambda x: B.T @ x, 60)
    assert abs(est - np.linalg.norm(B, 2)) < 1e-9 * 10
    A = gaussian((60, 60), 3)
    rel = relative_error(lambda x: A @ x, lambda x: A.T @ x, lambda x: 1.001 * (A @ x),
                         lambda x: 1.001 * (A.T @ x), 60)
    assert abs(rel - 0.001) < 1e-6


def test_check_shape_rejects_infeasible():
    with pytest.raises(ValueError):
        check_shape(1024, 10, 30, 64)            # leaf 64 > s - r
    with pytest.raises(ValueError):
        check_shape(1024, 10, 25, 16)            # s < 3r
    with pytest.raises(ValueError):
        check_shape(100, 10, 30, 8)              # leaves of 6-7 rows < r
    with pytest.raises(ValueError):
        check_shape(40, 3, 30, 64)               # single node with N > s
    check_shape(1024, 10, 30, 16)


# ---- planted mistakes: each must be caught by a pin above ---------------------------------

def _bad_node_step_drop_term(Om, Ps, Yt, Zt, r):
    P, Q = oc.null(Om, r), oc.null(Ps, r)
    U, V = oc.col(Yt @ P, r), oc.col(Zt @ Q, r)
    I = np.eye(Om.shape[0])
    return U, V, (I - U @ U.T) @ Yt @ oc.pinv(Om)             # second term of D dropped


def _bad_node_step_first_columns(Om, Ps, Yt, Zt, r):
    from oracle.linalg import full_q, householder_qr
    def first_null(B):                                         # first, not last, columns of Q
        refl, _ = householder_qr(B.T)
        return full_q(refl, B.shape[1])[:, :r]
    P, Q = first_null(Om), first_null(Ps)
    U, V = oc.col(Yt @ P, r), oc.col(Zt @ Q, r)
    I = np.eye(Om.shape[0])
    D = (I - U @ U.T) @ Yt @ oc.pinv(Om) + U @ U.T @ ((I - V @ V.T) @ Zt @ oc.pinv(Ps)).T
    return U, V, D


def _bad_merge_sign(Om, Ps, Yt, Zt, U, V, D, a, b):
    o, p, y, z = _GOOD_MERGE(Om, Ps, Yt, Zt, U, V, D, a, b)
    y = np.vstack([U[a].T @ (Yt[a] + D[a] @ Om[a]), U[b].T @ (Yt[b] + D[b] @ Om[b])])
    return o, p, y, z


def _bad_merge_transpose(Om, Ps, Yt, Zt, U, V, D, a, b):
    o, p, y, z = _GOOD_MERGE(Om, Ps, Yt, Zt, U, V, D, a, b)
    z = np.vstack([V[a].T @ (Zt[a] - D[a] @ Ps[a]), V[b].T @ (Zt[b] - D[b] @ Ps[b])])
    return o, p, y, z


def _bad_merge_swap_bases(Om, Ps, Yt, Zt, U, V, D, a, b):
    o, p, y, z = _GOOD_MERGE(Om, Ps, Yt, Zt, U, V, D, a, b)
    p = np.vstack([V[a].T @ Ps[a], V[b].T @ Ps[b]])            # Psi reduced with V, not U
    return o, p, y, z


@pytest.mark.parametrize("target,bad", [
    ("node_step", _bad_node_step_drop_term),
    ("node_step", _bad_node_step_first_columns),
    ("merge", _bad_merge_sign),
    ("merge", _bad_merge_transpose),
    ("merge", _bad_merge_swap_bases),
])
def test_planted_mistakes_are_caught(monkeypatch, target, bad):
    monkeypatch.setattr(oc, target, bad)
    errs = [_recovery_error(*case) for case in OVERSAMPLED[:2]]
    assert max(errs) > 1e-6


def test_planted_apply_transpose_mistake_is_caught(monkeypatch):
    g = exact_hbs(97, 10, 3, 3)
    A = g.dense()
    F = _generator_factors(g)
    X = gaussian((97, 2), 1)
    F.D = {t: d.T for t, d in F.D.items()}                      # forgets D -> D^* somewhere
    assert not np.allclose(oa.apply(F, X), A @ X, atol=1e-6)

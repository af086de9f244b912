"""Algorithm 2 ("Compressing an HBS matrix") -- oracle side.

Test infrastructure only (see ``oracle/__init__.py``).

Input: test matrices Omega, Psi (N x s) and samples Y = A Omega, Z = A^* Psi (Section 4,
opening paragraph), the rank r = k + p and the leaf threshold m. Output: the telescoping
factorization of Section 3.3 -- U_tau, V_tau, D_tau for every node on levels 1..L and D for
the root -- in the canonical form of Eq. (define_d_tau), so U_tau^* D_tau V_tau = 0.

The sweep follows Algorithm 2 level by level, finest first:
* leaf blocks are row slices of Omega, Psi, Y, Z (Section 4.1);
* a parent stacks its children's reduced test and sample matrices, Eq. (omega_tau_and_y_tau),
  with Psi and Z built "analogously" as Algorithm 2 spells out: Psi uses U, Z uses V and D^*;
* on levels l > 0: P = null(Omega_tau, r), Q = null(Psi_tau, r) (Section 4.1),
  U = col(Y_tau P, r) (Eq. u_tau_formula), V = col(Z_tau Q, r) (Eq. v_tau_formula),
  D_tau by Eq. (d_tau_formula);
* at the root: D = Y_tau Omega_tau^dagger (Section 4.3).

Feasibility (Section 4 asks for s >= max(r + m, 3r)): the nullspace of every leaf block must
hold r vectors (leaf size <= s - r), every leaf must have at least r rows for ``col``, and the
parent blocks (2r rows) need s >= 3r. With L = 0 the root is the only node and D = Y Omega^dagger
is exact only when N <= s. Infeasible shapes raise ValueError.
"""

from dataclasses import dataclass, field

import numpy as np

from .linalg import col, null, pinv
from .tree import build_tree, children, level_nodes


@dataclass
class HBSFactors:
    """Telescoping factorization of Section 3.3 (node ids as in Fig. 1)."""
    N: int
    r: int
    L: int
    offsets: list
    sizes: list
    U: dict = field(default_factory=dict)
    V: dict = field(default_factory=dict)
    D: dict = field(default_factory=dict)


def check_shape(N, r, s, leaf_max):
    """Raise ValueError unless (N, r, s, leaf_max) admits Algorithm 2; return (L, offsets, sizes)."""
    if min(N, r, s, leaf_max) < 1:
        raise ValueError("N, r, s and leaf_max must be positive")
    L, offsets, sizes = build_tree(N, leaf_max)
    if L == 0:
        if N > s:
            raise ValueError("single-node tree needs N <= s")
        return L, offsets, sizes
    leaves = sizes[2 ** L: 2 ** (L + 1)]
    if min(leaves) < r:
        raise ValueError("a leaf has fewer than r rows")
    if max(leaves) + r > s:
        raise ValueError("s < leaf size + r: leaf nullspace too small")
    if s < 3 * r:
        raise ValueError("s < 3r: parent nullspace too small")
    return L, offsets, sizes


def node_step(Om, Ps, Yt, Zt, r):
    """U_tau, V_tau, D_tau of one non-root node (Algorithm 2, "Compute blocks", l > 0)."""
    P = null(Om, r)
    Q = null(Ps, r)
    U = col(Yt @ P, r)
    V = col(Zt @ Q, r)
    n = Om.shape[0]
    I = np.eye(n)
    D = (I - U @ U.T) @ Yt @ pinv(Om) + U @ U.T @ ((I - V @ V.T) @ Zt @ pinv(Ps)).T
    return U, V, D


def merge(Om, Ps, Yt, Zt, U, V, D, a, b):
    """Test and sample blocks of a parent from children a, b (Eq. omega_tau_and_y_tau)."""
    Om_t = np.vstack([V[a].T @ Om[a], V[b].T @ Om[b]])
    Ps_t = np.vstack([U[a].T @ Ps[a], U[b].T @ Ps[b]])
    Y_t = np.vstack([U[a].T @ (Yt[a] - D[a] @ Om[a]), U[b].T @ (Yt[b] - D[b] @ Om[b])])
    Z_t = np.vstack([V[a].T @ (Zt[a] - D[a].T @ Ps[a]), V[b].T @ (Zt[b] - D[b].T @ Ps[b])])
    return Om_t, Ps_t, Y_t, Z_t


def compress(Omega, Psi, Y, Z, r, leaf_max, keep_blocks=False):
    """Algorithm 2. Returns HBSFactors (and, with keep_blocks, the per-node Omega/Psi/Y/Z)."""
    Omega, Psi, Y, Z = (np.asarray(x, dtype=np.float64) for x in (Omega, Psi, Y, Z))
    N, s = Omega.shape
    if Psi.shape != (N, s) or Y.shape != (N, s) or Z.shape != (N, s):
        raise ValueError("Omega, Psi, Y, Z must all be N x s")
    L, offsets, sizes = check_shape(N, r, s, leaf_max)
    F = HBSFactors(N=N, r=r, L=L, offsets=offsets, sizes=sizes)
    Om, Ps, Yt, Zt = {}, {}, {}, {}
    for level in range(L, -1, -1):
        for tau in level_nodes(level):
            if level == L:
                rows = slice(offsets[tau], offsets[tau] + sizes[tau])
                Om[tau], Ps[tau], Yt[tau], Zt[tau] = Omega[rows], Psi[rows], Y[rows], Z[rows]
            else:
                a, b = children(tau)
                Om[tau], Ps[tau], Yt[tau], Zt[tau] = merge(Om, Ps, Yt, Zt, F.U, F.V, F.D, a, b)
            if level > 0:
                F.U[tau], F.V[tau], F.D[tau] = node_step(Om[tau], Ps[tau], Yt[tau], Zt[tau], r)
            else:
                F.D[tau] = Yt[tau] @ pinv(Om[tau])
    if keep_blocks:
        return F, {"Omega": Om, "Psi": Ps, "Y": Yt, "Z": Zt}
    return F

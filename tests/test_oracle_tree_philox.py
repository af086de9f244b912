"""Pins for the oracle's tree (Section 3.1) and counter-based Gaussian generator."""

import os

import numpy as np
import pytest
from scipy import stats

from conftest import GOLDEN
from oracle import philox
from oracle.tree import build_tree, tree_depth


def _read(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_tree_matches_fig1_worked_example():
    rows = _read("fig1_tree.txt")
    kv = {r[0]: int(r[1]) for r in rows if len(r) == 2}
    L, off, sz = build_tree(kv["N"], kv["leaf_max"])
    assert L == kv["L"]
    for r in rows:
        if len(r) == 3:
            tau, first, last = map(int, r)
            assert off[tau] + 1 == first and off[tau] + sz[tau] == last


@pytest.mark.parametrize("N", [1, 2, 3, 7, 31, 64, 100, 400, 1000, 1023, 1025, 4097])
@pytest.mark.parametrize("leaf_max", [1, 5, 16, 64, 100])
def test_tree_partition_and_closed_form(N, leaf_max):
    L, off, sz = build_tree(N, leaf_max)
    # depth: ceil(N / 2^L) <= leaf_max < ceil(N / 2^(L-1))
    assert -(-N // 2 ** L) <= leaf_max
    if L > 0:
        assert -(-N // 2 ** (L - 1)) > leaf_max
    for level in range(L + 1):
        nodes = range(2 ** level, 2 ** (level + 1))
        # sizes on a level are floor or ceil of N / 2^level (closed form of repeated ceil splits)
        assert {sz[t] for t in nodes} <= {N // 2 ** level, -(-N // 2 ** level)}
        # the level partitions [0, N) into contiguous, ordered pieces
        pos = 0
        for t in nodes:
            assert off[t] == pos
            pos += sz[t]
        assert pos == N
    for t in range(1, 2 ** L):
        assert sz[2 * t] == -(-sz[t] // 2)         # left child takes ceil(n/2)


def test_tree_depth_brute_force():
    for N in range(1, 300):
        for m in (1, 3, 8, 17):
            L = tree_depth(N, m)
            assert L == next(l for l in range(64) if -(-N // 2 ** l) <= m)


def test_philox_known_answers():
    for r in _read("philox4x32_10_kat.txt"):
        w = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*(np.array([v], dtype=np.uint64) for v in w[:4]), w[4], w[5])
        assert [int(o[0]) for o in out] == w[6:]


def test_gaussian_layout_and_box_muller_identity():
    N, s, seed = 37, 11, 12345
    G = philox.gaussian_matrix(N, s, 0, seed)
    # rows drawn separately agree bit for bit with the full draw (counter = element pair index)
    assert np.array_equal(philox.gaussian_matrix(N, s, 0, seed, rows=[5, 36, 0]), G[[5, 36, 0]])
    # Box-Muller: the two normals of one pair satisfy z0^2 + z1^2 = -2 ln u1
    e = np.arange(0, N * s - 1, 2)
    z0, z1 = G.ravel()[e], G.ravel()[e + 1]
    x0, x1, _, _ = philox.philox4x32_10(e // 2, np.zeros_like(e), np.zeros_like(e),
                                        np.zeros_like(e), seed & 0xFFFFFFFF, seed >> 32)
    u1 = philox._uniform52(x0, x1)
    assert np.allclose(z0 ** 2 + z1 ** 2, -2 * np.log(u1), rtol=1e-13)
    # streams differ
    assert not np.array_equal(G, philox.gaussian_matrix(N, s, 1, seed))


def test_gaussian_distribution():
    z = philox.gaussian_matrix(4000, 50, 0, 7).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # neighbouring entries (same Philox output) are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.01

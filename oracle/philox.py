"""Gaussian test matrices Omega, Psi (Algorithm 2, first block; Section 2.3 step 2) -- oracle side.

Test infrastructure only (see ``oracle/__init__.py``).

The paper asks for i.i.d. standard Gaussian entries and fixes no generator. Both the oracle and
the GPU path implement one counter-based generator from its published definition, so that any
entry can be regenerated anywhere from (seed, stream, index):

* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
  1, 2, 3", SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; each round multiplies counter
  words 0 and 2 by the constants 0xD2511F53 and 0xCD9E8D57, and mixes the high halves with the
  other two words and the key; the key is bumped by the Weyl constants 0x9E3779B9 and
  0xBB67AE85 between rounds.
* Box-Muller (Box & Muller, 1958) turns each 4-word output into two normals.

Layout of one N x s test matrix, row-major element e = i*s + j, pair p = e // 2:
  counter = (p mod 2^32, p div 2^32, stream, 0), key = (seed mod 2^32, seed div 2^32)
  u1 = (hi52(x0, x1) + 1/2) 2^-52,  u2 = (hi52(x2, x3) + 1/2) 2^-52
       where hi52(a, b) is the top 52 bits of the 64-bit word a*2^32 + b
  rho = sqrt(-2 ln u1);  element 2p = rho cos(2 pi u2),  element 2p + 1 = rho sin(2 pi u2).
Stream 0 draws Omega, stream 1 draws Psi.
"""

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of 32-bit counter words (held in uint64); returns 4 word arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        prod0 = M0 * c0                      # < 2^64: exact in uint64
        prod1 = M1 * c2
        hi0, lo0 = prod0 >> np.uint64(32), prod0 & MASK32
        hi1, lo1 = prod1 >> np.uint64(32), prod1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def _uniform52(a, b):
    """(top 52 bits of a*2^32 + b, plus 1/2) * 2^-52: exactly representable, strictly in (0, 1)."""
    word = (a << np.uint64(32)) | b
    top = (word >> np.uint64(12)).astype(np.float64)        # < 2^52: exact
    return (top + 0.5) * 2.0 ** -52


def gaussian_pairs(pair_index, stream, seed):
    """Two standard normals per pair index (Box-Muller on one Philox output)."""
    p = np.asarray(pair_index, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(p & MASK32, p >> np.uint64(32),
                                   np.full_like(p, stream), np.zeros_like(p),
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = _uniform52(x0, x1)
    u2 = _uniform52(x2, x3)
    rho = np.sqrt(-2.0 * np.log(u1))
    return rho * np.cos(2.0 * np.pi * u2), rho * np.sin(2.0 * np.pi * u2)


def gaussian_matrix(N, s, stream, seed, rows=None):
    """Rows ``rows`` (default all) of the N x s test matrix drawn from (seed, stream)."""
    rows = np.arange(N, dtype=np.int64) if rows is None else np.asarray(rows, dtype=np.int64)
    e = (rows[:, None] * s + np.arange(s, dtype=np.int64)[None, :]).ravel()
    z0, z1 = gaussian_pairs((e // 2).astype(np.uint64), stream, seed)
    out = np.where(e % 2 == 0, z0, z1)
    return out.reshape(len(rows), s)


def gaussian_test_matrices(N, s, seed):
    """(Omega, Psi), both N x s (Algorithm 2: "Form Gaussian random test matrices")."""
    return gaussian_matrix(N, s, 0, seed), gaussian_matrix(N, s, 1, seed)

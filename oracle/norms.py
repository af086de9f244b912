"""Accuracy metric of Section 5 -- oracle side.

Test infrastructure only (see ``oracle/__init__.py``).

The paper estimates ||B|| for B in {A, A~ - A} by 20 steps of power iteration on B^* B from a
random start: v_i = B^* B (v_{i-1} / ||v_{i-1}||), ||B|| ~ sqrt(||v_20||). The start vector is
drawn from a seeded Gaussian (the paper does not fix it).
"""

import numpy as np


def power_norm(apply_B, apply_Bt, N, steps=20, seed=0):
    """Operator-norm estimate of B from 20 power steps (Section 5)."""
    v = np.random.default_rng(seed).standard_normal(N)
    for _ in range(steps):
        v = apply_Bt(apply_B(v / np.linalg.norm(v)))
    return float(np.sqrt(np.linalg.norm(v)))


def relative_error(apply_A, apply_At, apply_Ah, apply_Aht, N, steps=20, seed=0):
    """||A~ - A|| / ||A|| with both norms by ``power_norm`` (Section 5)."""
    num = power_norm(lambda x: apply_Ah(x) - apply_A(x), lambda x: apply_Aht(x) - apply_At(x),
                     N, steps, seed)
    den = power_norm(apply_A, apply_At, N, steps, seed)
    return num / den

"""Checks of the synthetic operators (inputs, not method arithmetic)."""

import numpy as np

from hbs_inputs import double_layer, log_kernel
from hbs_inputs.generators import _curve_geometry


def test_double_layer_gauss_law_and_diagonal_limit():
    # Gauss's law for the double layer on a closed curve: the kernel integrates to -1/2 for the
    # 1/(2 pi) normalization, so -1/4 with the 1/(4 pi) constant used; the trapezoid rule on this
    # smooth periodic curve is exact to rounding. The diagonal is the kernel's smooth limit.
    N = 2048
    A = double_layer(N)
    K = A - 0.5 * np.eye(N)
    assert np.allclose(K.sum(axis=1), -0.25, atol=1e-12)
    # the diagonal value is the limit of the neighbours: their mismatch falls like h^2
    def mismatch(n):
        Kn = double_layer(n) - 0.5 * np.eye(n)
        w = _curve_geometry(n)[4]
        i = np.arange(1, n - 1)
        kd = np.diag(Kn)[i] / w[i]
        nb = 0.5 * (Kn[i, i - 1] / w[i - 1] + Kn[i, i + 1] / w[i + 1])
        return np.max(np.abs(kd - nb))
    ratio = mismatch(2048) / mismatch(1024)
    assert 0.2 < ratio < 0.3


def test_log_kernel_symmetric_zero_diagonal():
    A = log_kernel(512)
    assert np.array_equal(A, A.T) and np.all(np.diag(A) == 0)

"""What the log-kernel workload allows a reduced precision to reach (readings A5/A22), measured
with the oracle alone (plain FP64, CPU).

The log kernel is compressed with r = k = 40 and s = 3r = 120: no oversampling beyond its
numerical rank, so the result moves under perturbations of the samples. Two kinds matter for
the mixed precisions:
* storing A in FP32 (each entry rounded to 2^-24): the oracle on the FP32-rounded A differs from
  the oracle on the FP64 A by ~15x the FP64 compression error at N = 4096 (6.9e-7 vs 4.5e-8;
  1.0e-6 at N = 8192, and it grows with N) -- so a workload that stores A in FP32 cannot meet
  a 1e-6 bar against the FP64 oracle whatever its arithmetic;
* product errors of 1e-10 (relative to sum |a_k b_k|), the size of the 5-digit tensor-core
  products: the result stays at the FP64 compression error.
"""

import numpy as np
import pytest

from hbs_inputs import gaussian, log_kernel
from oracle.apply import apply
from oracle.compress import compress


@pytest.fixture(scope="module")
def case():
    N, r, s, leaf = 4096, 40, 120, 64
    A = log_kernel(N)
    Om, Ps, X = gaussian((N, s), 1), gaussian((N, s), 2), gaussian((N, 16), 3)
    run = lambda Y, Z: apply(compress(Om, Ps, Y, Z, r, leaf), X)
    ref = run(A @ Om, A.T @ Ps)
    AX = A @ X
    err64 = np.linalg.norm(ref - AX) / np.linalg.norm(AX)
    return dict(A=A, Om=Om, Ps=Ps, run=run, ref=ref, AX=AX, err64=err64, N=N)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_fp32_storage_of_A_moves_the_result_past_the_fp64_error(case):
    A32 = case["A"].astype(np.float32).astype(np.float64)
    o32 = case["run"](A32 @ case["Om"], A32.T @ case["Ps"])
    assert case["err64"] < 1e-7
    assert _rel(o32, case["ref"]) > 5 * case["err64"]


def test_products_at_1e_10_keep_the_fp64_error(case):
    A, Om, Ps, N = case["A"], case["Om"], case["Ps"], case["N"]
    rng = np.random.default_rng(7)
    Y = A @ Om + 1e-10 * rng.standard_normal(Om.shape) * (np.abs(A) @ np.abs(Om)) / np.sqrt(N)
    Z = A.T @ Ps + 1e-10 * rng.standard_normal(Ps.shape) * (np.abs(A).T @ np.abs(Ps)) / np.sqrt(N)
    o = case["run"](Y, Z)
    assert _rel(o, case["AX"]) <= 3 * case["err64"]
    assert _rel(o, case["ref"]) <= 3 * case["err64"]

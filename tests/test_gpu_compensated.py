"""The compensated mixed precision (HBS_PREC_MIXED_COMPENSATED) against the FP64 oracle.

Products: the FP64 A and test matrices written as 5 exact 8-bit digits per entry (one exponent
per 64 x 64 block of A, read transposed for A^*, and per 64-row window of a test matrix), the
15 digit pairs with i + j <= 4 multiplied on the tensor cores with
exactly representable FP32 sums. Each entry is represented to 2^-39 of its block's largest
magnitude and each dropped pair weighs at most 6 * 2^-38 of the product of the block maxima, so
an output entry errs by ~2^-36 times sum_k (max|a| max|b|) over its windows; for these inputs the
block maxima are within ~30x of the typical entries, hence the bounds below: 1e-9 of
sum_k |a_k b_k| per entry, 1e-10 relative Frobenius (measured 0.8e-12 .. 2.7e-12 per entry,
7.4e-12 .. 2.0e-11 Frobenius).

Sweep: the LQ of each test block and the bases in FP64, D_tau and the merges in double-float
(FP32 pairs, ~2^-48 per operation). Factors are held to the FP64 bar, 1e-10, against the oracle
(measured 3e-13 .. 1.3e-12 on these shapes; the plain FP32 finish gives 1e-5 .. 5e-5).

Pipelines (products + sweep), against the oracle run on the same FP64 A: exact-HBS matrices
with oversampling to 1e-8 (measured 1.1e-9: the product error, amplified ~1e2 by the
compression), and the log kernel to the 1e-6 target that this precision exists for (measured
1.8e-8 at N = 2048, 6e-8 at N = 8192, where the FP64 GPU path itself differs from the oracle by
2e-8 and 8e-8: reading A22, the log kernel's compression moves by about its own error under any
perturbation).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import exact_hbs, gaussian, log_kernel
from oracle import apply as oapply
from oracle.compress import compress as ocompress
from oracle.sample import sample as osample

pytestmark = pytest.mark.gpu

CMP = 4   # HBS_PREC_MIXED_COMPENSATED


@pytest.fixture(scope="module")
def hb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    import paper_2205_02990_gb300 as hb
    from paper_2205_02990_gb300 import hbs
    if not os.path.exists(hbs._LIB_PATH):
        from paper_2205_02990_gb300.build import build
        build()
    hb.load()
    assert hb.HBS_PREC_MIXED_COMPENSATED == CMP
    return hb


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,s,kind", [(4099, 130, "log"), (2048, 120, "gauss"), (200, 7, "gauss"),
                                      (1, 3, "gauss"), (1000, 256, "log")])
def test_compensated_products(hb, N, s, kind):
    A = log_kernel(N) if kind == "log" else gaussian((N, N), 3 + N)
    Om, Ps = gaussian((N, s), 1), gaussian((N, s), 2)
    Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(2))
    hb.hbs_sample_products(dev(A), s, dev(Om), dev(Ps), Y, Z, precision=CMP)
    hb.hbs_sample_sync()
    Yr, Zr = A @ Om, A.T @ Ps
    assert rel(host(Y), Yr) <= 1e-10 and rel(host(Z), Zr) <= 1e-10
    assert np.max(np.abs(host(Y) - Yr) / (np.abs(A) @ np.abs(Om))) <= 1e-9
    assert np.max(np.abs(host(Z) - Zr) / (np.abs(A).T @ np.abs(Ps))) <= 1e-9


def test_compensated_products_graded_rows_and_columns(hb):
    """Rows and columns of A graded over 2^-20 .. 2^20: one exponent per 64 x 64 block keeps
    the normwise bound (a numpy model of the rounding to 2^-39 of each block's largest entry
    gives 2.1e-11), while entries far below their block's largest lose relative accuracy (the
    same model: 0.44 of sum_k |a_k b_k| at worst). HBS_PREC_FP64_TC, one exponent per row (per
    column for A^*) and window, keeps the per-entry bound on the same matrix."""
    N, s = 1000, 64
    rng = np.random.default_rng(7)
    dr, dc = 2.0 ** rng.integers(-20, 21, N), 2.0 ** rng.integers(-20, 21, N)
    A = dr[:, None] * gaussian((N, N), 11) * dc[None, :]
    Om, Ps = gaussian((N, s), 1), gaussian((N, s), 2)
    Yr, Zr = A @ Om, A.T @ Ps
    for precision in (CMP, 3):
        Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(2))
        hb.hbs_sample_products(dev(A), s, dev(Om), dev(Ps), Y, Z, precision=precision)
        hb.hbs_sample_sync()
        assert rel(host(Y), Yr) <= 1e-10 and rel(host(Z), Zr) <= 1e-10
        if precision == 3:
            assert np.max(np.abs(host(Y) - Yr) / (np.abs(A) @ np.abs(Om))) <= 1e-12
            assert np.max(np.abs(host(Z) - Zr) / (np.abs(A).T @ np.abs(Ps))) <= 1e-12


def _worst_factor(hb, h, F, blk, L, item=0):
    """Worst relative error of U, V, D over every node; D_tau against the magnitude that enters
    it, ||Y_tau Omega_tau^+|| (a leaf of exactly r rows has D_tau = 0 up to rounding), as in
    test_gpu_parity.py."""
    from oracle.linalg import pinv
    worst = 0.0
    for t in range(1, 2 ** (L + 1)):
        U, V, D = hb.hbs_get_node(h, t, item=item)
        scale = max(np.linalg.norm(F.D[t]), np.linalg.norm(blk["Y"][t] @ pinv(blk["Omega"][t])))
        worst = max(worst, np.linalg.norm(D.numpy() - F.D[t]) / scale)
        if t > 1:
            worst = max(worst, rel(U.numpy(), F.U[t]), rel(V.numpy(), F.V[t]))
    return worst


@pytest.mark.parametrize("N,r,s,leaf", [(2048, 40, 120, 64), (1024, 10, 30, 16), (777, 12, 40, 26),
                                        (3000, 16, 48, 32), (129, 4, 12, 8),
                                        # upper nodes of 100 rows: their double-float tiles exceed
                                        # shared memory, those heights run the FP64 finish
                                        (4096, 50, 150, 64)])
def test_compensated_sweep_random_inputs(hb, N, r, s, leaf):
    x = [gaussian((N, s), 7 * N + i) for i in range(4)]
    F, blk = ocompress(*x, r, leaf, keep_blocks=True)
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, *[dev(v) for v in x])], precision=CMP)
    hb.hbs_sync_status(h)
    assert _worst_factor(hb, h, F, blk, F.L) <= 1e-10
    h.free()


def test_compensated_batch_of_uneven_trees(hb):
    # The second height holds 80 nodes of the four trees (up to 80 rows, s = 120): one side-kernel
    # CTA per (node, side) at two CTAs per SM, whose double-float rows take the reflectors in pairs.
    cases = [(1024, 10, 30, 16), (777, 12, 40, 26), (129, 4, 12, 8), (2048, 40, 120, 64)]
    probs, refs = [], []
    for j, (N, r, s, leaf) in enumerate(cases):
        x = [gaussian((N, s), 600 + 4 * j + i) for i in range(4)]
        refs.append(ocompress(*x, r, leaf, keep_blocks=True))
        probs.append(hb.Problem(N, r, s, leaf, *[dev(v) for v in x]))
    h = hb.hbs_compress(probs, precision=CMP)
    hb.hbs_sync_status(h)
    for j, (F, blk) in enumerate(refs):
        assert _worst_factor(hb, h, F, blk, F.L, item=j) <= 1e-10, j
    h.free()


def _pipeline(hb, A, N, r, s, leaf, seed, X):
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(dev(A), s, seed, Om, Ps, Y, Z, precision=CMP)
    hb.hbs_sample_sync()
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)], precision=CMP)
    hb.hbs_sync_status(h)
    out, outT = (torch.empty((N, X.shape[1]), dtype=torch.float64, device="cuda") for _ in range(2))
    hb.hbs_apply(h, dev(X), out)
    hb.hbs_apply(h, dev(X), outT, trans=True)
    torch.cuda.synchronize()
    h.free()
    return host(out), host(outT)


@pytest.mark.parametrize("N,k,r,s,leaf", [(4096, 8, 12, 36, 24), (1000, 6, 9, 27, 18)])
def test_compensated_pipeline_exact_hbs(hb, N, k, r, s, leaf):
    A = exact_hbs(N, leaf, k, 11).dense()
    X = gaussian((N, 8), 5)
    out, outT = _pipeline(hb, A, N, r, s, leaf, 99, X)
    Fo = ocompress(*osample(A, N, s, 99), r, leaf)
    assert rel(out, A @ X) <= 1e-8 and rel(outT, A.T @ X) <= 1e-8
    assert rel(out, oapply.apply(Fo, X)) <= 1e-8
    assert rel(outT, oapply.apply(Fo, X, trans=True)) <= 1e-8


def test_compensated_pipeline_log_kernel_meets_target(hb):
    N, r, s, leaf = 2048, 40, 120, 64
    A = log_kernel(N)
    X = gaussian((N, 8), 6)
    out, _ = _pipeline(hb, A, N, r, s, leaf, 5, X)
    ref = oapply.apply(ocompress(*osample(A, N, s, 5), r, leaf), X)
    assert rel(out, ref) <= 1e-6                       # the mixed-precision target
    e_gpu, e_orc = rel(out, A @ X), rel(ref, A @ X)
    assert e_gpu <= 3 * e_orc and e_orc <= 3 * e_gpu   # and the oracle's own accuracy

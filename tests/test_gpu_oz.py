"""FP64-class sampling by exact digit products on the tensor cores (HBS_PREC_FP64_TC).

Y = A Omega and Z = A^* Psi (Algorithm 2, first block) are formed from six balanced 8-bit digits
per FP64 entry (one exponent per 64-wide block), with the digit-pair products whose sums the
tensor core's FP32 accumulator holds exactly. The error budget per term is ~2^-47 of the block
maxima (digit representation and the dropped pairs), plus double-float accumulation over 2048
indices; FP64 itself carries 2^-53 per term and K u in the worst case. Tolerances:

* sampled entries against the exactly rounded dot product (TwoProduct + math.fsum):
  |y - y_exact| <= 2^-40 sum_k |a_k b_k| (the FP64 product's worst-case bound for K = 4096 is
  2^-41 of the same sum);
* relative Frobenius error of Y and Z against numpy's FP64 product: 1e-13;
* rows scaled over 2^-30 .. 2^30: every row to 1e-12 of its own norm (per-row exponents);
* factors of the FP64 sweep on these samples: the FP64 bars of the parity tests (1e-11 recovery
  of exactly-HBS matrices, 1e-10 against the oracle).
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import exact_hbs, gaussian, log_kernel, log_kernel_rows, log_kernel_torch
from oracle import apply as oapply
from oracle import philox
from oracle.compress import compress as ocompress
from oracle.sample import sample as osample

pytestmark = pytest.mark.gpu

TC = 3          # HBS_PREC_FP64_TC


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
    assert hb.HBS_PREC_FP64_TC == TC
    return hb


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def exact_dot(a, b):
    """sum_k a_k b_k correctly rounded: Dekker's TwoProduct (Veltkamp splitting) + fsum."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    p = a * b
    c = 134217729.0                                  # 2^27 + 1

    def split(x):
        t = c * x
        hi = t - (t - x)
        return hi, x - hi

    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return math.fsum(np.concatenate([p, e]))


CMP = 4   # HBS_PREC_MIXED_COMPENSATED: 5 digits, one exponent per 64 x 64 block of A
# relative Frobenius bound of the scaled products per precision (5 digits: ~2^-36 per entry)
SCALED_BOUND = {TC: 1e-13, CMP: 1e-10}


def sample_tc(hb, A, s, seed, precision=TC):
    N = A.shape[0]
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(dev(A), s, seed, Om, Ps, Y, Z, precision=precision)
    hb.hbs_sample_sync()
    return [host(x) for x in (Om, Ps, Y, Z)]


def check_entries(A, B, C, rows, cols, trans=False):
    for i in rows:
        a = A[:, i] if trans else A[i]
        for j in cols:
            ex = exact_dot(a, B[:, j])
            bound = 2.0 ** -40 * float(np.abs(a) @ np.abs(B[:, j]))
            assert abs(C[i, j] - ex) <= bound, (i, j, C[i, j], ex, bound)


@pytest.mark.parametrize("N,s,kind", [(1000, 30, "log"), (777, 120, "gauss"), (64, 7, "log"),
                                      (1, 3, "gauss"), (4099, 130, "log"), (2048, 256, "gauss"),
                                      (130, 33, "gauss")])
def test_digit_products_match_fp64(hb, N, s, kind):
    A = log_kernel(N) if kind == "log" else gaussian((N, N), 3 * N)
    seed = 77 + N
    Om, Ps, Y, Z = sample_tc(hb, A, s, seed)
    Omr, Psr, Yr, Zr = osample(A, N, s, seed)
    assert np.abs(Om - Omr).max() <= 1e-13 and np.abs(Ps - Psr).max() <= 1e-13
    assert rel(Y, Yr) <= 1e-13 and rel(Z, Zr) <= 1e-13
    rng = np.random.default_rng(N)
    rows = rng.choice(N, min(N, 6), replace=False)
    cols = rng.choice(s, min(s, 4), replace=False)
    check_entries(A, Omr, Y, rows, cols)
    check_entries(A, Psr, Z, rows, cols, trans=True)


def test_rows_and_columns_over_a_wide_range(hb):
    # A = D1 G D2 with D1, D2 powers of two in 2^-30 .. 2^30, a zero row, a zero column and a
    # zero 64 x 64 block: every row of Y (and of Z = A^* Psi) keeps its own relative accuracy.
    N, s = 1500, 40
    rng = np.random.default_rng(5)
    d1 = np.exp2(rng.integers(-30, 31, N).astype(np.float64))
    d2 = np.exp2(rng.integers(-30, 31, N).astype(np.float64))
    A = d1[:, None] * gaussian((N, N), 8) * d2[None, :]
    A[17] = 0.0
    A[:, 900] = 0.0
    A[128:192, 640:704] = 0.0
    Om, Ps, Y, Z = sample_tc(hb, A, s, 3)
    Yr, Zr = A @ Om, A.T @ Ps
    assert np.all(Y[17] == 0.0) and np.all(Z[900] == 0.0)
    for C, Cr in ((Y, Yr), (Z, Zr)):
        nz = np.linalg.norm(Cr, axis=1) > 0
        err = np.linalg.norm(C - Cr, axis=1)[nz] / np.linalg.norm(Cr, axis=1)[nz]
        assert err.max() <= 1e-12, err.max()
    check_entries(A, Om, Y, [0, 17, 130, 1499], [0, 39])


@pytest.mark.parametrize("precision", [TC, CMP])
def test_scale_far_from_one(hb, precision):
    # the whole FP64 exponent range: A ~ 2^-600 and A ~ 2^+600 give the scaled products
    N, s = 300, 20
    G = gaussian((N, N), 4)
    for e in (-600, 600):
        A = np.ldexp(G, e)
        Om, Ps, Y, Z = sample_tc(hb, A, s, 9, precision)
        assert rel(np.ldexp(Y, -e), G @ Om) <= SCALED_BOUND[precision]
        assert rel(np.ldexp(Z, -e), G.T @ Ps) <= SCALED_BOUND[precision]


@pytest.mark.parametrize("precision", [TC, CMP])
def test_subnormal_operator(hb, precision):
    # A ~ 2^-1040: every entry subnormal (~34 significant bits). Its digits need left shifts of
    # the mantissa by up to ~21 bits; the products land on the subnormal grid (2^-1074), so they
    # match the exact product to its rounding, 2^-1074 per entry (~1e-10 relative here).
    N, s = 300, 20
    A = np.ldexp(gaussian((N, N), 6), -1040)
    Gs = np.ldexp(A, 1040)                             # exactly A's values, scaled up
    Om, Ps, Y, Z = sample_tc(hb, A, s, 10, precision)
    assert rel(np.ldexp(Y, 1040), Gs @ Om) <= 1e-8
    assert rel(np.ldexp(Z, 1040), Gs.T @ Ps) <= 1e-8


@pytest.mark.parametrize("precision", [TC, CMP])
def test_non_finite_entry_is_reported(hb, precision):
    N, s = 200, 12
    A = gaussian((N, N), 2)
    A[3, 150] = np.nan
    X = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
    hb.hbs_sample(dev(A), s, 1, *X, precision=precision)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample_sync()
    assert e.value.code == -5
    hb.hbs_sample_sync()                                 # the status was cleared


def test_digit_products_need_a_dense_fp64_operator(hb):
    N, s = 64, 8
    X = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample(torch.zeros((N, N), dtype=torch.float32, device="cuda"), s, 1, *X, precision=TC)
    assert e.value.code == -8
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample(lambda t, x, o: o.copy_(x), s, 1, *X, precision=TC, N=N)
    assert e.value.code == -8


@pytest.mark.parametrize("precision", [TC, CMP])
def test_repeated_calls_are_bit_identical(hb, precision):
    N, s = 1000, 30
    A = log_kernel(N)
    first = sample_tc(hb, A, s, 4, precision)
    second = sample_tc(hb, A, s, 4, precision)
    for a, b in zip(first, second):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("N,k,r,s,leaf", [(400, 5, 8, 24, 16), (1000, 6, 9, 27, 18),
                                          (4096, 8, 12, 36, 24)])
def test_pipeline_exact_hbs(hb, N, k, r, s, leaf):
    g = exact_hbs(N, leaf, k, 11)
    A = g.dense()
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(dev(A), s, 99, Om, Ps, Y, Z, precision=TC)
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)], precision=TC)
    hb.hbs_sync_status(h)
    hb.hbs_sample_sync()
    X = torch.eye(N, dtype=torch.float64, device="cuda")
    Out = torch.empty_like(X)
    hb.hbs_apply(h, X, Out)
    torch.cuda.synchronize()
    At = host(Out)
    assert rel(At, A) <= 1e-11
    F = ocompress(*osample(A, N, s, 99), r, leaf)
    assert rel(At, oapply.dense(F)) <= 1e-10


def test_full_size_log_kernel_sampled_entries(hb):
    # the bench's workload: log kernel N = 32768, s = 120, A resident in HBM (8.6 GB)
    N, r, s, leaf, seed = 32768, 40, 120, 64, 220502990 + 200
    A = log_kernel_torch(N, "cuda")
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(A, s, seed, Om, Ps, Y, Z, precision=TC)
    hb.hbs_sample_sync()
    rows = np.random.default_rng(1).choice(N, 4, replace=False)
    Omr = philox.gaussian_matrix(N, s, 0, seed)
    Psr = philox.gaussian_matrix(N, s, 1, seed)
    Arows = log_kernel_rows(N, rows)                     # A is symmetric: rows = columns
    Yh, Zh = host(Y[rows]), host(Z[rows])
    assert rel(Yh, Arows @ Omr) <= 1e-13 and rel(Zh, Arows @ Psr) <= 1e-13
    for ii, i in enumerate(rows):
        for j in (0, 57, 119):
            for C, B in ((Yh, Omr), (Zh, Psr)):
                ex = exact_dot(Arows[ii], B[:, j])
                assert abs(C[ii, j] - ex) <= 2.0 ** -40 * float(np.abs(Arows[ii]) @ np.abs(B[:, j]))
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)], precision=TC)
    hb.hbs_sync_status(h)
    Xp = torch.randn((N, 4), dtype=torch.float64, device="cuda",
                     generator=torch.Generator("cuda").manual_seed(1))
    Out = torch.empty_like(Xp)
    hb.hbs_apply(h, Xp, Out)
    assert rel(host(Out), host(A @ Xp)) <= 1e-5
    del A

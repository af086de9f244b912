"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same inputs.

Tolerances (relative Frobenius unless stated):
* test matrices: |z_gpu - z_oracle| <= 1e-13 per entry -- same Philox words, libm vs CUDA
  log/sqrt/sincos differ by ulps only;
* samples Y, Z: 1e-12 -- FP64 products with K = N terms in another summation order;
* factors U, V, D and reconstructions on well-conditioned inputs: 1e-10, the FP64 bar. The
  oracle itself moves by ~1e-13 under 1e-16 perturbations of its inputs on these cases;
* inputs where the method itself is ill-conditioned (exact rank with no oversampling, or the
  log kernel, where a 1e-16 change of Y moves the result by 3e-9 .. 3e-8 in the oracle) are
  compared by their accuracy against A instead (see the individual tests).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import exact_hbs, gaussian, log_kernel, log_kernel_rows, log_kernel_torch
from oracle import apply as oapply
from oracle import philox
from oracle.compress import compress as ocompress
from oracle.sample import sample as osample
from oracle.tree import build_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_02990_gb300 as hb
    from paper_2205_02990_gb300 import hbs
    import os
    if not os.path.exists(hbs._LIB_PATH):
        from paper_2205_02990_gb300.build import build
        build()
    hb.load()
    return hb


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_compress(hb, N, r, s, leaf, Om, Ps, Y, Z):
    tens = [t if isinstance(t, torch.Tensor) else dev(t) for t in (Om, Ps, Y, Z)]
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, *tens)])
    hb.hbs_sync_status(h)
    h.keep = tens
    return h


def gpu_dense(hb, h, N, trans=False):
    X = torch.eye(N, dtype=torch.float64, device="cuda")
    Out = torch.empty_like(X)
    hb.hbs_apply(h, X, Out, trans=trans)
    torch.cuda.synchronize()
    return host(Out)


# ---- test matrices ---------------------------------------------------------------------

@pytest.mark.parametrize("N,s,stream,seed", [(37, 11, 0, 12345), (1000, 120, 1, 220503090),
                                             (3, 1, 0, 2 ** 40 + 7), (513, 30, 1, 0)])
def test_gaussian_matches_oracle(hb, N, s, stream, seed):
    out = torch.empty((N, s), dtype=torch.float64, device="cuda")
    hb.hbs_draw_gaussian(N, s, stream, seed, out)
    ref = philox.gaussian_matrix(N, s, stream, seed)
    assert np.abs(host(out) - ref).max() <= 1e-13


# ---- sampling ------------------------------------------------------------------------------

@pytest.mark.parametrize("N,s,kind", [(1000, 30, "log"), (777, 120, "gauss"), (64, 7, "log"),
                                      (1, 3, "gauss"), (4099, 130, "log")])
def test_sample_dense_matches_oracle(hb, N, s, kind):
    A = log_kernel(N) if kind == "log" else gaussian((N, N), N)
    seed = 1000 + N
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(dev(A), s, seed, Om, Ps, Y, Z)
    Omr, Psr, Yr, Zr = osample(A, N, s, seed)
    assert np.abs(host(Om) - Omr).max() <= 1e-13
    assert np.abs(host(Ps) - Psr).max() <= 1e-13
    assert rel(host(Y), Yr) <= 1e-12 and rel(host(Z), Zr) <= 1e-12


# ---- the sweep on well-conditioned (random) inputs: every factor of every node --------------

RANDOM_CASES = [(1024, 10, 30, 16), (1000, 7, 21, 14), (2048, 40, 120, 64), (777, 12, 40, 26),
                (20, 3, 26, 32), (30, 5, 20, 15), (3000, 16, 48, 32), (129, 4, 12, 8)]


def factor_errors(hb, h, F, blk, nodes, item=0):
    """Worst relative error of U, V, D over ``nodes``. D_tau is measured against the magnitude
    that enters it, ||Y_tau Omega_tau^+||: where a leaf has exactly r rows, U and V span
    everything and D_tau is zero up to rounding."""
    from oracle.linalg import pinv
    worst, where = 0.0, None
    for t in nodes:
        U, V, D = hb.hbs_get_node(h, t, item=item)
        scale = max(np.linalg.norm(F.D[t]), np.linalg.norm(blk["Y"][t] @ pinv(blk["Omega"][t])))
        errs = {"D": np.linalg.norm(D.numpy() - F.D[t]) / scale}
        if t > 1:
            errs["U"] = rel(U.numpy(), F.U[t])
            errs["V"] = rel(V.numpy(), F.V[t])
        for k, e in errs.items():
            if e > worst:
                worst, where = e, (t, k)
    return worst, where


@pytest.mark.parametrize("case", RANDOM_CASES)
def test_sweep_random_inputs_all_factors(hb, case):
    N, r, s, leaf = case
    Om, Ps, Y, Z = (gaussian((N, s), 7 * N + i) for i in range(4))
    F, blk = ocompress(Om, Ps, Y, Z, r, leaf, keep_blocks=True)
    h = gpu_compress(hb, N, r, s, leaf, Om, Ps, Y, Z)
    L, off, size = hb.hbs_tree(h)
    Lo, offo, sizeo = build_tree(N, leaf)
    assert (L, off, size) == (Lo, offo[1:], sizeo[1:])
    worst, where = factor_errors(hb, h, F, blk, range(1, 2 ** (L + 1)))
    assert worst <= 1e-10, (worst, where)


# ---- whole pipeline on exactly-HBS matrices ------------------------------------------------

def pipeline(hb, A, N, r, s, leaf, seed):
    Ad = dev(A)
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(Ad, s, seed, Om, Ps, Y, Z)
    return gpu_compress(hb, N, r, s, leaf, Om, Ps, Y, Z)


@pytest.mark.parametrize("N,k,r,s,leaf", [(400, 5, 8, 24, 16), (1000, 6, 9, 27, 18),
                                          (4096, 8, 12, 36, 24), (257, 4, 7, 21, 14)])
def test_exact_hbs_recovery_and_parity(hb, N, k, r, s, leaf):
    g = exact_hbs(N, leaf, k, 11)
    A = g.dense()
    h = pipeline(hb, A, N, r, s, leaf, 99)
    At = gpu_dense(hb, h, N)
    assert rel(At, A) <= 1e-11                                   # exact recovery (r > k)
    F = ocompress(*osample(A, N, s, 99), r, leaf)
    assert rel(At, oapply.dense(F)) <= 1e-10                     # parity with the oracle
    AtT = gpu_dense(hb, h, N, trans=True)
    assert rel(AtT, A.T) <= 1e-11                                # Algorithm 1 with A^*


def test_exact_hbs_without_oversampling(hb):
    # exact-HBS, N = 1024, k = r = 10, s = 30, leaf 16 (p = 0). The oracle's own output moves by
    # ~3e-9 under 1e-16 changes of Y here, so both sides are held to the recovery bound.
    N, k, s, leaf = 1024, 10, 30, 16
    g = exact_hbs(N, leaf, k, 1)
    A = g.dense()
    h = pipeline(hb, A, N, k, s, leaf, 7)
    At = gpu_dense(hb, h, N)
    F = ocompress(*osample(A, N, s, 7), k, leaf)
    Ao = oapply.dense(F)
    assert rel(At, A) <= 1e-7 and rel(Ao, A) <= 1e-7
    assert rel(At, Ao) <= 1e-7


def test_log_kernel_accuracy_matches_oracle(hb):
    # log kernel, r = 40, s = 120, leaf 64 at N = 2048: not exactly HBS; the result is only
    # determined to the compression error, so GPU and oracle must reach the same accuracy.
    N, r, s, leaf = 2048, 40, 120, 64
    A = log_kernel(N)
    h = pipeline(hb, A, N, r, s, leaf, 5)
    At = gpu_dense(hb, h, N)
    Ao = oapply.dense(ocompress(*osample(A, N, s, 5), r, leaf))
    e_gpu, e_orc = rel(At, A), rel(Ao, A)
    assert e_gpu <= 1e-6 and e_orc <= 1e-6
    assert e_gpu <= 3 * e_orc and e_orc <= 3 * e_gpu
    assert rel(At, Ao) <= 3 * e_orc


def test_single_node_tree(hb):
    N, s = 20, 26
    A = gaussian((N, N), 4)
    h = pipeline(hb, A, N, 3, s, 32, 3)
    _, _, D = hb.hbs_get_node(h, 1)
    assert rel(D.numpy(), A) <= 1e-12


def test_apply_columns_match_dense(hb):
    N, k, r, s, leaf = 1000, 6, 9, 27, 18
    A = exact_hbs(N, leaf, k, 2).dense()
    h = pipeline(hb, A, N, r, s, leaf, 4)
    for c in (1, 3, 130):
        X = gaussian((N, c), c)
        Out = torch.empty((N, c), dtype=torch.float64, device="cuda")
        hb.hbs_apply(h, dev(X), Out)
        assert rel(host(Out), A @ X) <= 1e-11


def test_execute_reuses_plan_with_new_inputs(hb):
    N, r, s, leaf = 1000, 7, 21, 14
    ins = [[gaussian((N, s), 50 * j + i) for i in range(4)] for j in range(2)]
    tens = [[dev(x) for x in grp] for grp in ins]
    h = hb.hbs_plan([hb.Problem(N, r, s, leaf, *tens[0])])
    for grp, t in zip(ins, tens):
        hb.hbs_execute(h, [hb.Problem(N, r, s, leaf, *t)])
        hb.hbs_sync_status(h)
        F = ocompress(*grp, r, leaf)
        _, _, D = hb.hbs_get_node(h, 5)
        assert rel(D.numpy(), F.D[5]) <= 1e-10


def test_batch_of_uneven_trees(hb):
    cases = [(1024, 10, 30, 16), (777, 12, 40, 26), (129, 4, 12, 8), (20, 3, 26, 32)]
    probs, refs = [], []
    for j, (N, r, s, leaf) in enumerate(cases):
        x = [gaussian((N, s), 900 + 4 * j + i) for i in range(4)]
        refs.append(ocompress(*x, r, leaf, keep_blocks=True))
        probs.append(hb.Problem(N, r, s, leaf, *[dev(v) for v in x]))
    h = hb.hbs_compress(probs)
    hb.hbs_sync_status(h)
    for j, (F, blk) in enumerate(refs):
        worst, where = factor_errors(hb, h, F, blk, range(1, 2 ** (F.L + 1)), item=j)
        assert worst <= 1e-10, (j, worst, where)
    # the side kernel as clusters sharing one factorization (ragged row ownership, CTAs without
    # rows where C > n) rounds exactly as the single-CTA form
    ref = [[hb.hbs_get_node(h, t, item=j) for t in range(1, 2 ** (F.L + 1))]
           for j, (F, _) in enumerate(refs)]
    H = len(hb.hbs_get_tuning(h))
    for tuning in ([-1] * H, [-2] * H, [-3] * H, [-8] * H):
        hb.hbs_set_tuning(h, tuning)
        hb.hbs_execute(h, probs)
        hb.hbs_sync_status(h)
        for j, (F, _) in enumerate(refs):
            for t, want in zip(range(1, 2 ** (F.L + 1)), ref[j]):
                got = hb.hbs_get_node(h, t, item=j)
                for a, b in zip(got, want):
                    assert (a is None and b is None) or torch.equal(a, b), (tuning, j, t)


def test_numeric_status_on_singular_block(hb):
    # Omega with a zero row has a zero pivot: the device flags HBS_ERR_NUMERIC (host-side
    # read of the status word; nothing faults)
    N, r, s, leaf = 64, 4, 12, 8
    Om = gaussian((N, s), 1)
    Om[3] = 0.0
    x = [Om] + [gaussian((N, s), i) for i in range(2, 5)]
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, *[dev(v) for v in x])])
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sync_status(h)
    assert e.value.code == -5


# ---- the full-size sampling workload (log kernel, N = 32768) -------------------------------

def test_full_size_log_kernel_sampled_parity(hb):
    N, r, s, leaf, seed = 32768, 40, 120, 64, 220502990 + 200
    A = log_kernel_torch(N, "cuda")
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(A, s, seed, Om, Ps, Y, Z)
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)])
    hb.hbs_sync_status(h)
    rows = np.random.default_rng(0).choice(N, 6, replace=False)
    Omr = philox.gaussian_matrix(N, s, 0, seed)
    Psr = philox.gaussian_matrix(N, s, 1, seed)
    Arows = log_kernel_rows(N, rows)                   # A is symmetric: rows = columns
    assert rel(host(Y[rows]), Arows @ Omr) <= 1e-12
    assert rel(host(Z[rows]), Arows @ Psr) <= 1e-12
    # properties of the factors on sampled nodes (Section 2.4, Eq. define_d_tau canonical form)
    for t in (2, 3, 100, 511, 512, 1023):
        U, V, D = (x.numpy() for x in hb.hbs_get_node(h, t))
        assert np.abs(U.T @ U - np.eye(r)).max() <= 1e-12
        assert np.abs(V.T @ V - np.eye(r)).max() <= 1e-12
        assert np.abs(U.T @ D @ V).max() <= 1e-10 * max(1.0, np.abs(D).max())
    # accuracy of the compressed operator on random probes (error of the method, ~1e-7 here)
    X = torch.randn((N, 4), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    Out = torch.empty_like(X)
    hb.hbs_apply(h, X, Out)
    assert rel(host(Out), host(A @ X)) <= 1e-5
    del A


def test_double_layer_accuracy_matches_oracle(hb):
    # the Section 5.1 boundary integral operator with the paper's r = 30, m = 60, s = 90
    from hbs_inputs import double_layer
    N, r, s, leaf = 2048, 30, 90, 60
    A = double_layer(N)
    h = pipeline(hb, A, N, r, s, leaf, 8)
    At = gpu_dense(hb, h, N)
    Ao = oapply.dense(ocompress(*osample(A, N, s, 8), r, leaf))
    e_gpu, e_orc = rel(At, A), rel(Ao, A)
    assert e_gpu <= 1e-6 and e_orc <= 1e-6
    assert e_gpu <= 3 * e_orc and e_orc <= 3 * e_gpu


def test_profile_sweep_times_every_phase_and_keeps_factors(hb):
    # hbs_profile_sweep re-runs the sweep with plain launches and events between them: one
    # time per (height, phase), and the factors it leaves are bit-identical (same inputs)
    N, r, s, leaf = 2048, 40, 120, 64
    x = [dev(gaussian((N, s), 40 + i)) for i in range(4)]
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, *x)])
    hb.hbs_sync_status(h)
    L = hb.hbs_tree(h)[0]
    before = [hb.hbs_get_node(h, t) for t in range(1, 2 ** (L + 1))]
    ms = hb.hbs_profile_sweep(h)
    hb.hbs_sync_status(h)
    assert len(ms) == L + 1
    for t, row in enumerate(ms):
        assert len(row) == 4 and all(v >= 0 for v in row)
        assert row[0] > 0                                  # every height runs the side kernel
        if t < L:
            assert min(row) > 0                            # and, below the root, all four
    after = [hb.hbs_get_node(h, t) for t in range(1, 2 ** (L + 1))]
    for a, b in zip(before, after):
        for u, v in zip(a, b):
            assert (u is None and v is None) or torch.equal(u, v)
    h.free()


def test_full_size_tree_every_factor_matches_oracle(hb):
    # The headline tree (N = 32768, r = 40, s = 120, leaf 64: 1023 nodes over 10 levels, the
    # same launches and tuned side shapes as the benchmark) on well-conditioned inputs, where the
    # factors are determined to rounding (the log kernel's are not: reading A22), so every U, V,
    # D of every node is held to the FP64 bar against the oracle.
    N, r, s, leaf = 32768, 40, 120, 64
    x = [gaussian((N, s), 5100 + i) for i in range(4)]
    F, blk = ocompress(*x, r, leaf, keep_blocks=True)
    tens = [dev(v) for v in x]
    h = hb.hbs_plan([hb.Problem(N, r, s, leaf, *tens)])
    hb.hbs_execute(h)
    hb.hbs_autotune(h)                                 # the benchmark's tuned shapes
    hb.hbs_execute(h)
    hb.hbs_sync_status(h)
    worst, where = factor_errors(hb, h, F, blk, range(1, 2 ** (F.L + 1)))
    assert worst <= 1e-10, (worst, where)
    h.free()


@pytest.mark.parametrize("precision", [0, 2, 4])
def test_autotune_keeps_factors_bit_identical(hb, precision):
    # hbs_autotune picks the side shape and the finish kernels' grids (merge chunk, D column
    # blocks) per height; every choice rounds alike, so the factors after a tuned execution are
    # bit-identical to the automatic ones
    N, r, s, leaf = 4096, 40, 120, 64
    x = [dev(gaussian((N, s), 70 + i)) for i in range(4)]
    h = hb.hbs_plan([hb.Problem(N, r, s, leaf, *x)], precision=precision)
    hb.hbs_execute(h)
    hb.hbs_sync_status(h)
    before = torch.empty(hb.hbs_factor_bytes(h) // 8, dtype=torch.float64, device="cuda")
    hb.hbs_copy_factors(h, before)
    hb.hbs_autotune(h)
    hb.hbs_execute(h)
    hb.hbs_sync_status(h)
    after = torch.empty_like(before)
    hb.hbs_copy_factors(h, after)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    h.free()

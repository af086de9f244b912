"""hbs_sample_execute: the leaves' test-block LQ on a second stream while the products run.

The LQ of a leaf's Omega_tau and Psi_tau depends on the test matrices alone (Section 2.4; the
single-view remark of Section 1: everything that needs only the test matrices can be done
before the operator is applied). hbs_sample_execute runs those factorizations (node_lq) on the
handle's own stream from the draws on, and the leaf level's side kernel copies them in instead
of recomputing them. The same instructions make them, so samples and factors must be
bit-identical to hbs_sample + hbs_execute, in every precision, with and without the captured
sweep graph, on repeated calls, and where the leaf level runs the cluster form (no overlap).
Accuracy against the oracle is that of the plain path (tested in test_gpu_parity.py and
test_gpu_compensated.py); one exact-HBS case is checked here end to end.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import exact_hbs, gaussian, log_kernel

pytestmark = pytest.mark.gpu

FP64, BF16X6, FP64_TC, CMP = 0, 2, 3, 4


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
    return hb


def dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def blocks(N, s):
    return [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]


def factors(hb, h):
    out = torch.empty(hb.hbs_factor_bytes(h) // 8, dtype=torch.float64, device="cuda")
    hb.hbs_copy_factors(h, out)
    torch.cuda.synchronize()
    return out


def plain(hb, A, N, r, s, leaf, seed, sample_prec, sweep_prec, graph=True):
    x = blocks(N, s)
    hb.hbs_sample(A, s, seed, *x, precision=sample_prec, N=N)
    h = hb.hbs_plan([hb.Problem(N, r, s, leaf, *x)], precision=sweep_prec)
    hb.hbs_set_graph(h, graph)
    hb.hbs_execute(h)
    hb.hbs_sync_status(h)
    hb.hbs_sample_sync()
    return h, x


def overlapped(hb, A, N, r, s, leaf, seed, sample_prec, sweep_prec, graph=True, calls=1):
    x = blocks(N, s)
    h = hb.hbs_plan([hb.Problem(N, r, s, leaf, *x)], precision=sweep_prec)
    hb.hbs_set_graph(h, graph)
    for _ in range(calls):
        hb.hbs_sample_execute(h, A, seed, precision=sample_prec, N=N)
    hb.hbs_sync_status(h)
    hb.hbs_sample_sync()
    return h, x


@pytest.mark.parametrize("sample_prec,sweep_prec", [(FP64, FP64), (FP64_TC, FP64_TC), (CMP, CMP),
                                                    (BF16X6, BF16X6), (BF16X6, FP64)])
@pytest.mark.parametrize("graph", [True, False])
def test_overlapped_leaf_lq_is_bit_identical(hb, sample_prec, sweep_prec, graph):
    N, r, s, leaf = 4096, 20, 60, 32                    # 128 leaves: one CTA per (leaf, side)
    A64 = log_kernel(N)
    A = dev(A64, torch.float32 if sample_prec == BF16X6 else torch.float64)
    h0, x0 = plain(hb, A, N, r, s, leaf, 11, sample_prec, sweep_prec, graph)
    h1, x1 = overlapped(hb, A, N, r, s, leaf, 11, sample_prec, sweep_prec, graph, calls=2)
    for a, b in zip(x0, x1):
        assert torch.equal(a, b)
    assert torch.equal(factors(hb, h0), factors(hb, h1))
    h0.free()
    h1.free()


def test_few_leaves_run_the_cluster_form_unchanged(hb):
    # 4 leaves of 64 rows: the leaf level runs the cluster side kernel, nothing is overlapped
    N, r, s, leaf = 256, 10, 80, 64
    A = dev(gaussian((N, N), 5))
    h0, _ = plain(hb, A, N, r, s, leaf, 3, FP64, FP64)
    h1, _ = overlapped(hb, A, N, r, s, leaf, 3, FP64, FP64)
    assert torch.equal(factors(hb, h0), factors(hb, h1))
    h0.free()
    h1.free()


def test_black_box_operator_exact_hbs_recovery(hb):
    # a callback operator (the black box of Algorithm 2): exact-HBS input, k = 6, r = 9
    N, k, r, s, leaf = 2000, 6, 9, 30, 20
    A = dev(exact_hbs(N, leaf, k, 21).dense())

    def fn(trans, X, Out):
        torch.matmul(A.T if trans else A, X, out=Out)

    h0, _ = plain(hb, fn, N, r, s, leaf, 8, FP64, FP64)
    h1, _ = overlapped(hb, fn, N, r, s, leaf, 8, FP64, FP64)
    assert torch.equal(factors(hb, h0), factors(hb, h1))
    I = torch.eye(N, dtype=torch.float64, device="cuda")
    out = torch.empty_like(I)
    hb.hbs_apply(h1, I, out)
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(out - A) / torch.linalg.norm(A))
    assert err <= 1e-11, err
    h0.free()
    h1.free()


def test_pinned_host_operator_is_bit_identical(hb):
    # A in page-locked host memory: the FP64 products stream it through the device in row
    # blocks on the caller's stream while the leaves' LQ runs on the handle's stream
    N, r, s, leaf = 4096, 20, 60, 32
    A = torch.as_tensor(log_kernel(N)).pin_memory()
    h0, x0 = plain(hb, A, N, r, s, leaf, 13, FP64, FP64)
    h1, x1 = overlapped(hb, A, N, r, s, leaf, 13, FP64, FP64, calls=2)
    for a, b in zip(x0, x1):
        assert torch.equal(a, b)
    assert torch.equal(factors(hb, h0), factors(hb, h1))
    h0.free()
    h1.free()


def test_sample_execute_argument_errors(hb):
    N, r, s, leaf = 512, 8, 30, 16
    x = blocks(N, s)
    y = blocks(N, s)
    A = dev(gaussian((N, N), 2))
    h2 = hb.hbs_plan([hb.Problem(N, r, s, leaf, *x), hb.Problem(N, r, s, leaf, *y)])
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample_execute(h2, A, 1, problems=h2.problems[:1])
    assert e.value.code == -1
    h2.free()
    h = hb.hbs_plan([hb.Problem(N, r, s, leaf, *x)])
    with pytest.raises(hb.HBSError) as e:                # the operator's N differs
        hb.hbs_sample_execute(h, dev(gaussian((N + 1, N + 1), 3)), 1)
    assert e.value.code == -1
    with pytest.raises(hb.HBSError) as e:                # digit products need a FP64 A
        hb.hbs_sample_execute(h, A.float(), 1, precision=FP64_TC)
    assert e.value.code == -8
    hb.hbs_sample_execute(h, A, 1)                       # the handle is still usable
    hb.hbs_sync_status(h)
    h.free()

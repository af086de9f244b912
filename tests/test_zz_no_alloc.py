"""hbs_apply_static: Algorithm 1 for callers that must not allocate device memory.

cudaMalloc synchronizes the device and fails when another allocator (a framework's caching
pool, say) already holds the GPU's memory, so latency-bound services and black-box operator
callbacks that apply a compressed matrix in the middle of someone else's stream cannot call
hbs_apply the first time it needs workspace. hbs_apply_static keeps its workspace and work list
in fixed arrays inside the library.

These tests call it through the C ABI on a fresh handle before any hbs_apply, twice in a row
(A, then A^*), and check each result against the existing entry point hbs_apply (1e-12, the
same kernel in the same order) and against the dense exactly-HBS matrix the handle recovered
(1e-11, the exact-recovery bar of test_gpu_parity.py); that a warm call takes no device memory;
and that requests beyond either fixed limit are refused before anything runs. This file is
collected last so that a stop at its first failure comes after every other test.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import exact_hbs, gaussian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2205_02990_gb300 as hb
    from paper_2205_02990_gb300 import hbs
    if not os.path.exists(hbs._LIB_PATH):
        from paper_2205_02990_gb300.build import build
        build()
    hb.load()
    return hb


def _compressed(hb, A, N, r, s, leaf, seed):
    Ad = torch.as_tensor(A, device="cuda")
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(Ad, s, seed, Om, Ps, Y, Z)
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)])
    hb.hbs_sync_status(h)
    h.keep = (Om, Ps, Y, Z)
    return h


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("N,k,r,s,leaf,c", [(1000, 6, 9, 27, 18, 3), (20, 3, 3, 26, 32, 2),
                                            (4096, 8, 12, 36, 24, 1)])
def test_static_apply_twice_matches_apply_and_dense(hb, N, k, r, s, leaf, c):
    A = exact_hbs(N, leaf, k, 5).dense()
    h = _compressed(hb, A, N, r, s, leaf, 5)
    Ad = torch.as_tensor(A, device="cuda")
    outs = []
    for call, (trans, seed) in enumerate([(False, 1), (True, 2)]):
        X = torch.as_tensor(gaussian((N, c), seed), device="cuda")
        out = torch.full_like(X, float("nan"))
        hb.hbs_apply_static(h, X, out, trans=trans)    # before any hbs_apply on this handle
        torch.cuda.synchronize()
        dense = (Ad.T if trans else Ad) @ X
        assert _rel(out, dense) <= 1e-11, (call, trans)
        outs.append((X, out, trans))
    for call, (X, out, trans) in enumerate(outs):
        ref = torch.empty_like(X)
        hb.hbs_apply(h, X, ref, trans=trans)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= 1e-12, (call, trans)
    h.free()


def test_static_apply_takes_no_device_memory(hb):
    N, k, r, s, leaf = 1000, 6, 9, 27, 18
    A = exact_hbs(N, leaf, k, 6).dense()
    h = _compressed(hb, A, N, r, s, leaf, 6)
    X = torch.as_tensor(gaussian((N, 4), 3), device="cuda")
    Out = torch.empty_like(X)
    hb.hbs_apply_static(h, X, Out)                     # warm: arrays set up on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for trans in (False, True, False):
        hb.hbs_apply_static(h, X, Out, trans=trans)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    h.free()


def test_static_apply_rejects_oversized_workspace(hb):
    N, k, r, s, leaf = 1000, 6, 9, 27, 18
    h = _compressed(hb, exact_hbs(N, leaf, k, 7).dense(), N, r, s, leaf, 7)
    c = 1000                                   # 2 (2^7 - 2) 9 c doubles > the fixed workspace
    X = torch.zeros((N, c), dtype=torch.float64, device="cuda")
    Out = torch.zeros_like(X)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_apply_static(h, X, Out)
    assert e.value.code == -8 and "exceeds" in str(e.value)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Out).item() == 0
    h.free()


def test_static_apply_rejects_oversized_work_list(hb):
    # N = 16384 with leaves of 2 rows: L = 13, 2^15 - 3 = 32765 node products > the fixed 16384
    # (the workspace, 2 (2^14 - 2) doubles for r = c = 1, is within its limit)
    N, r, s, leaf = 16384, 1, 3, 2
    x = [torch.as_tensor(gaussian((N, s), 30 + i), device="cuda") for i in range(4)]
    h = hb.hbs_plan([hb.Problem(N, r, s, leaf, *x)])
    assert hb.hbs_tree(h)[0] == 13
    X = torch.ones((N, 1), dtype=torch.float64, device="cuda")
    Out = torch.zeros_like(X)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_apply_static(h, X, Out)
    assert e.value.code == -8 and "node products" in str(e.value)
    torch.cuda.synchronize()
    assert torch.count_nonzero(Out).item() == 0
    h.free()

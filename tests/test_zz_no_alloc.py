"""hbs_apply_static: Algorithm 1 for callers that must not allocate device memory.

cudaMalloc synchronizes the device and fails when another allocator already holds the GPU's
memory, so latency-bound services and black-box operator callbacks cannot call hbs_apply the
first time it needs workspace. hbs_apply_static keeps workspace and work list in fixed arrays
inside the library. These tests call it through the C ABI twice in a row and compare with
hbs_apply, and check that an oversized request is refused before anything runs.
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


def _compressed(hb, N, k, r, s, leaf, seed):
    A = exact_hbs(N, leaf, k, seed).dense()
    Ad = torch.as_tensor(A, device="cuda")
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    hb.hbs_sample(Ad, s, seed, Om, Ps, Y, Z)
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)])
    hb.hbs_sync_status(h)
    h.keep = (Om, Ps, Y, Z)
    return h


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("N,k,r,s,leaf,c", [(1000, 6, 9, 27, 18, 3), (20, 3, 3, 26, 32, 2)])
def test_static_apply_matches_apply_twice(hb, N, k, r, s, leaf, c):
    h = _compressed(hb, N, k, r, s, leaf, 5)
    for call, (trans, seed) in enumerate([(False, 1), (True, 2)]):
        X = torch.as_tensor(gaussian((N, c), seed), device="cuda")
        ref = torch.empty_like(X)
        out = torch.full_like(X, float("nan"))
        hb.hbs_apply(h, X, ref, trans=trans)
        hb.hbs_apply_static(h, X, out, trans=trans)
        torch.cuda.synchronize()
        assert _rel(out, ref) <= 1e-12, (call, trans)
    h.free()


def test_static_apply_rejects_oversized_request(hb):
    h = _compressed(hb, 1000, 6, 9, 27, 18, 7)
    c = 1000                                   # 2 (2^7 - 2) 9 c doubles > the fixed workspace
    X = torch.zeros((1000, c), dtype=torch.float64, device="cuda")
    Out = torch.zeros_like(X)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_apply_static(h, X, Out)
    assert e.value.code == -8 and "exceeds" in str(e.value)
    assert torch.count_nonzero(Out).item() == 0
    h.free()

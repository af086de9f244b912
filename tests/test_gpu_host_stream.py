"""FP64 products with A in page-locked host memory, streamed through the device in row blocks.

Y = A Omega and Z = A^* Psi (Algorithm 2, first block) from a pinned host A must equal the
products from a device A up to summation order (row blocks change the split of the reduction):
1e-13 relative against the device result and the FP64 parity bar of 1e-12 against the oracle.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import gaussian, log_kernel
from oracle.sample import sample as osample

pytestmark = pytest.mark.gpu


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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def pinned(A, pad):
    N = A.shape[0]
    buf = torch.empty((N, N + pad), dtype=torch.float64, pin_memory=True)
    view = buf[:, :N]
    view.copy_(torch.as_tensor(A))
    return view


@pytest.mark.parametrize("N,s,pad,kind", [(1000, 30, 0, "log"), (777, 120, 5, "gauss"),
                                          (1, 3, 0, "gauss"), (4099, 130, 3, "log"),
                                          (2048, 64, 0, "gauss")])
def test_host_streamed_products(hb, N, s, pad, kind):
    A = log_kernel(N) if kind == "log" else gaussian((N, N), 2 * N + 1)
    seed = 500 + N
    Ah = pinned(A, pad)
    assert Ah.is_pinned() and Ah.stride(0) == N + pad
    out = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
    hb.hbs_sample(Ah, s, seed, *out)
    ref = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
    hb.hbs_sample(torch.as_tensor(A, device="cuda"), s, seed, *ref)
    torch.cuda.synchronize()
    Om, Ps, Y, Z = (t.cpu().numpy() for t in out)
    _, _, Yd, Zd = (t.cpu().numpy() for t in ref)
    assert rel(Y, Yd) <= 1e-13 and rel(Z, Zd) <= 1e-13
    _, _, Yr, Zr = osample(A, N, s, seed)
    assert rel(Y, Yr) <= 1e-12 and rel(Z, Zr) <= 1e-12


def test_host_stream_repeats_bit_identically(hb):
    N, s = 1500, 40
    Ah = pinned(gaussian((N, N), 9), 0)
    runs = []
    for _ in range(2):
        out = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
        hb.hbs_sample(Ah, s, 3, *out)
        torch.cuda.synchronize()
        runs.append([t.cpu() for t in out])
    for a, b in zip(*runs):
        assert torch.equal(a, b)


def test_pageable_host_memory_is_rejected(hb):
    from paper_2205_02990_gb300 import hbs
    N, s = 64, 8
    A = np.ascontiguousarray(gaussian((N, N), 1))         # pageable host memory
    op = hbs._Operator(N=N, dtype=hbs.HBS_F64, A=A.ctypes.data, lda=N, fn=hbs.MATMAT_FN(), user=None)
    X = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
    rc = hbs.load().hbs_sample_products(ctypes.byref(op), s, 0, *[ctypes.c_void_p(t.data_ptr()) for t in X],
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1

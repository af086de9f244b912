"""Mixed-precision sampling on the tensor cores against the FP64 oracle.

A is stored in FP32; the oracle multiplies the same FP32 values held exactly in FP64. The
bound for each mode follows from its arithmetic: bf16x3 keeps ~16 significant bits of each
operand (relative error ~2^-16 = 1.5e-5 per product), so Y and Z are held to 5e-5; bf16x6
keeps ~24 bits, and its accumulator truncates at full magnitude only in the 4 leading-pair MMAs
of each 64-column step before the step is drained into a double-float sum (~4 x 2^-25 = 1.2e-7
per step), so Y and Z are held to 1e-6 relative Frobenius error.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import gaussian, log_kernel
from oracle.sample import sample as osample

pytestmark = pytest.mark.gpu

BOUND = {1: 5e-5, 2: 1e-6}


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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("N,s,kind", [(1000, 30, "log"), (4099, 120, "log"), (2048, 130, "gauss"),
                                      (200, 7, "gauss"), (4096, 256, "log")])
def test_mixed_sampling_matches_oracle(hb, prec, N, s, kind):
    A32 = (log_kernel(N) if kind == "log" else gaussian((N, N), N)).astype(np.float32)
    A64 = A32.astype(np.float64)                       # the exact values the GPU multiplies
    seed = 77 + N
    Om, Ps, Y, Z = (torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4))
    lda = (N + 3) // 4 * 4                              # row pitch must be a multiple of 16 bytes
    Ad = torch.zeros((N, lda), dtype=torch.float32, device="cuda")[:, :N]
    Ad.copy_(torch.as_tensor(A32))
    hb.hbs_sample(Ad, s, seed, Om, Ps, Y, Z, precision=prec)
    hb.hbs_sample_sync()
    Omr, Psr, Yr, Zr = osample(A64, N, s, seed)
    assert np.abs(Om.cpu().numpy() - Omr).max() <= 1e-13
    ey, ez = rel(Y.cpu().numpy(), Yr), rel(Z.cpu().numpy(), Zr)
    assert ey <= BOUND[prec] and ez <= BOUND[prec], (ey, ez)


def test_mixed_rejects_unaligned_rows(hb):
    N, s = 99, 8
    A = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    X = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample(A, s, 1, *X, precision=2)
    assert e.value.code == -8


def test_mixed_rejects_fp64_operator(hb):
    N, s = 64, 8
    A = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    X = [torch.empty((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample(A, s, 1, *X, precision=2)
    assert e.value.code == -8

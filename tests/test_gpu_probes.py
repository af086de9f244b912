"""The library's measurement probes (no counterpart in the paper; they give the bench its
denominators and the digit GEMM's issue bound): plausible values on a GB300.

* hbs_probe_peaks: DFMA and FFMA chains on every SM, TFLOP/s; GB300 has 2 DFMA and 128 FFMA
  per clock per SM (1.26 and 80.5 TFLOP/s at 2070 MHz), so the measured rates sit below those;
* hbs_probe_dmma: the FP64 tensor instruction, about the DFMA rate on GB300;
* hbs_probe_mma_issue: cycles per M = N = 128, K = 16 FP16 MMA issued by one thread; the tensor
  pipe takes 64 cycles per such MMA when nothing else runs, and no less beside other work.
"""

import math

import pytest

torch = pytest.importorskip("torch")

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


def test_pipe_probes(hb):
    fp64, fp32 = hb.hbs_probe_peaks()
    assert 0.3 <= fp64 <= 1.3, fp64
    assert 20.0 <= fp32 <= 82.0, fp32
    dmma = hb.hbs_probe_dmma()
    assert 0.3 <= dmma <= 1.3, dmma


def test_mma_issue_probe(hb):
    c = hb.hbs_probe_mma_issue()
    assert all(math.isfinite(v) and v > 0 for v in c.values()), c
    assert 56.0 <= c["alone"] <= 96.0, c                 # the pipe's 64 cycles, little overhead
    assert c["fp32_all_schedulers"] >= 0.95 * c["alone"], c
    assert c["fp32_other_schedulers"] >= 0.95 * c["alone"], c

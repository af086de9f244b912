"""Device status words through the C ABI: timeouts are reported, and a timeout left by one run
never cuts a later run short.

A bounded device-side wait that gives up sets the timeout bit of its status word and the abort
flag of its run (so the run's other waits end too). These tests put that state in place with the
test-only export hbs_test_inject_status -- no kernel is made to time out, nothing hangs or
faults -- and check that (i) hbs_sync_status / hbs_sample_sync return HBS_ERR_TIMEOUT once and
then clear, and (ii) the next compression or sampling, with the stale abort flag still set when
it is queued, waits normally: its factors match the oracle at the FP64 bar (1e-10, as in
test_gpu_parity.py) and its products are bit-identical to a run without the stale flag.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import gaussian, log_kernel
from oracle.compress import compress as ocompress

pytestmark = pytest.mark.gpu

TIMEOUT = 2


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


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def worst_factor_error(hb, h, F, L):
    worst = 0.0
    for t in range(1, 2 ** (L + 1)):
        U, V, D = hb.hbs_get_node(h, t)
        worst = max(worst, np.linalg.norm(D.numpy() - F.D[t]) / np.linalg.norm(F.D[t]))
        if t > 1:
            worst = max(worst, np.linalg.norm(U.numpy() - F.U[t]) / np.linalg.norm(F.U[t]),
                        np.linalg.norm(V.numpy() - F.V[t]) / np.linalg.norm(F.V[t]))
    return worst


@pytest.mark.parametrize("graph", [True, False])
def test_sweep_timeout_reported_and_next_run_unaffected(hb, graph):
    # N = 2048, r = 40, s = 120, leaf 64: the upper heights run the cluster form of the side
    # kernel, whose per-row waits are the abortable ones
    N, r, s, leaf = 2048, 40, 120, 64
    x = [gaussian((N, s), 4100 + i) for i in range(4)]
    F = ocompress(*x, r, leaf)
    probs = [hb.Problem(N, r, s, leaf, *[dev(v) for v in x])]
    h = hb.hbs_plan(probs)
    hb.hbs_set_graph(h, graph)
    hb.hbs_execute(h)
    hb.hbs_sync_status(h)
    L = hb.hbs_tree(h)[0]
    assert worst_factor_error(hb, h, F, L) <= 1e-10
    # a timeout recorded with no kernel running is reported once, then cleared
    hb.hbs_test_inject_status(h, TIMEOUT)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sync_status(h)
    assert e.value.code == -6
    hb.hbs_sync_status(h)
    # a stale timeout (report bit and abort flag) when the next run is queued: that run still
    # waits for every row and matches the oracle; the stale report is read afterwards
    zeros = torch.zeros(hb.hbs_factor_bytes(h) // 8, dtype=torch.float64, device="cuda")
    hb.hbs_load_factors(h, zeros)                      # the previous factors are gone
    hb.hbs_test_inject_status(h, TIMEOUT)
    hb.hbs_execute(h)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sync_status(h)
    assert e.value.code == -6
    assert worst_factor_error(hb, h, F, L) <= 1e-10
    hb.hbs_execute(h)
    hb.hbs_sync_status(h)                              # nothing left over
    h.free()


@pytest.mark.parametrize("precision", ["bf16x6", "digits"])
def test_sampling_timeout_reported_and_next_run_unaffected(hb, precision):
    N, s = 1000, 40
    A = log_kernel(N)
    if precision == "bf16x6":
        Ad = torch.as_tensor(A.astype(np.float32), device="cuda")
        prec = hb.HBS_PREC_MIXED_BF16X6
    else:
        Ad = dev(A)
        prec = hb.HBS_PREC_FP64_TC
    Om, Ps = dev(gaussian((N, s), 1)), dev(gaussian((N, s), 2))
    Y1, Z1 = (torch.zeros((N, s), dtype=torch.float64, device="cuda") for _ in range(2))
    hb.hbs_sample_products(Ad, s, Om, Ps, Y1, Z1, precision=prec)
    hb.hbs_sample_sync()
    hb.hbs_test_inject_status(None, TIMEOUT)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample_sync()
    assert e.value.code == -6
    hb.hbs_sample_sync()
    # stale abort flag when the next products are queued: they still run to the end
    hb.hbs_test_inject_status(None, TIMEOUT)
    Y2, Z2 = (torch.zeros((N, s), dtype=torch.float64, device="cuda") for _ in range(2))
    hb.hbs_sample_products(Ad, s, Om, Ps, Y2, Z2, precision=prec)
    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample_sync()
    assert e.value.code == -6
    assert torch.equal(Y1, Y2) and torch.equal(Z1, Z2)
    hb.hbs_sample_sync()

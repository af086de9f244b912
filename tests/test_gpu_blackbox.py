"""Black-box operators, batches, graph replay and tuning, through the C ABI.

A known telescoping factorization (the exact-HBS generator of Section 3.2, in the form of
Section 3.3) is loaded into a handle and applied by Algorithm 1; that handle is then the black
box (Section 1: A is reachable only through products) for the sampling of Algorithm 2.
"""

import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from hbs_inputs import exact_hbs, gaussian, pack_telescoping
from oracle import apply as oapply
from oracle.compress import compress as ocompress
from oracle.sample import sample as osample

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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def zeros(N, s):
    return [torch.zeros((N, s), dtype=torch.float64, device="cuda") for _ in range(4)]


def generator_handle(hb, gens, leafs):
    """Handle holding the generators' telescoping factors (never executed)."""
    probs = []
    for g, leaf in zip(gens, leafs):
        s = max(3 * g.k, (g.sizes[2 ** g.L] if g.L else g.N) + g.k, g.N if g.L == 0 else 0)
        probs.append(hb.Problem(g.N, g.k, s, leaf, *zeros(g.N, s)))
    h = hb.hbs_plan(probs)
    packed = np.concatenate([pack_telescoping(g) for g in gens])
    hb.hbs_load_factors(h, torch.as_tensor(packed, device="cuda"))
    return h


@pytest.mark.parametrize("N,leaf,k", [(400, 16, 8), (97, 10, 5), (64, 8, 4), (20, 32, 3), (1000, 24, 12)])
def test_loaded_factors_apply_matches_blockwise_assembly(hb, N, leaf, k):
    g = exact_hbs(N, leaf, k, 5)
    A = g.dense()
    h = generator_handle(hb, [g], [leaf])
    X = torch.eye(N, dtype=torch.float64, device="cuda")
    Out = torch.empty_like(X)
    hb.hbs_apply(h, X, Out)
    torch.cuda.synchronize()
    assert rel(Out.cpu().numpy(), A) <= 1e-12
    hb.hbs_apply(h, X, Out, trans=True)
    torch.cuda.synchronize()
    assert rel(Out.cpu().numpy(), A.T) <= 1e-12


@pytest.mark.parametrize("N,leaf,k", [(3000, 30, 10), (150, 256, 4)])
def test_skinny_apply_matches_wide_bitwise(hb, N, leaf, k):
    # 1 .. 4 right-hand-side columns take the skinny path (one thread per row, factors staged
    # k-major); wider ones the general path. Both add the products in the same order, so a
    # column applied alone equals the same column of an 8-column apply bit for bit. N = 150 with
    # leaf 256 is a single 150 x 150 block, beyond the skinny path's 128 rows: it falls back.
    g = exact_hbs(N, leaf, k, 7)
    A = g.dense()
    h = generator_handle(hb, [g], [leaf])
    X = torch.as_tensor(np.random.default_rng(N).standard_normal((N, 8)), device="cuda")
    for trans in (False, True):
        wide = torch.empty_like(X)
        hb.hbs_apply(h, X, wide, trans=trans)
        for c in (1, 3, 4):
            Xs = X[:, :c].contiguous()
            out = torch.empty_like(Xs)
            hb.hbs_apply(h, Xs, out, trans=trans)
            assert torch.equal(out, wide[:, :c]), (trans, c)
        ref = (A.T if trans else A) @ X.cpu().numpy()
        assert rel(wide.cpu().numpy(), ref) <= 1e-12


def test_repeated_apply_reuses_work_list_correctly(hb):
    # repeated calls with the same buffers reuse the uploaded work list: new contents of X, new
    # factors loaded into the handle, another direction and another stream must all show
    N, leaf, k = 900, 20, 6
    g1, g2 = exact_hbs(N, leaf, k, 21), exact_hbs(N, leaf, k, 22)
    h = generator_handle(hb, [g1], [leaf])
    X = torch.empty((N, 2), dtype=torch.float64, device="cuda")
    Out = torch.empty_like(X)
    rng = np.random.default_rng(5)
    for g, trans in ((g1, False), (g1, False), (g1, True), (g2, False), (g2, True)):
        if g is g2:
            hb.hbs_load_factors(h, torch.as_tensor(pack_telescoping(g2), device="cuda"))
        X.copy_(torch.as_tensor(rng.standard_normal((N, 2))))
        hb.hbs_apply(h, X, Out, trans=trans)
        A = g.dense()
        ref = (A.T if trans else A) @ X.cpu().numpy()
        assert rel(Out.cpu().numpy(), ref) <= 1e-12
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        hb.hbs_apply(h, X, Out)
    side.synchronize()
    assert rel(Out.cpu().numpy(), g2.dense() @ X.cpu().numpy()) <= 1e-12
    # the batched apply reuses its list the same way
    g3 = exact_hbs(500, 16, 5, 23)
    hbb = generator_handle(hb, [g1, g3], [leaf, 16])
    Xs = [torch.empty((g.N, 3), dtype=torch.float64, device="cuda") for g in (g1, g3)]
    Outs = [torch.empty_like(x) for x in Xs]
    for trans in (False, False, True, True):
        for x in Xs:
            x.copy_(torch.as_tensor(rng.standard_normal(tuple(x.shape))))
        hb.hbs_apply_batch(hbb, Xs, Outs, trans=trans)
        for g, x, o in zip((g1, g3), Xs, Outs):
            A = g.dense()
            assert rel(o.cpu().numpy(), (A.T if trans else A) @ x.cpu().numpy()) <= 1e-12


def test_skinny_batched_apply_matches_wide_bitwise(hb):
    # a batch whose items all have 2 columns takes the grouped skinny kernel; items with unequal
    # column counts the general one: both equal the wide single-item applies bit for bit
    gens = [exact_hbs(1200, 24, 8, 11), exact_hbs(700, 20, 6, 12), exact_hbs(90, 128, 5, 13)]
    h = generator_handle(hb, gens, [24, 20, 128])
    rng = np.random.default_rng(3)
    Xw = [torch.as_tensor(rng.standard_normal((g.N, 6)), device="cuda") for g in gens]
    for trans in (False, True):
        wide = [torch.empty_like(x) for x in Xw]
        for j, x in enumerate(Xw):
            hb.hbs_apply(h, x, wide[j], item=j, trans=trans)
        for widths in ((2, 2, 2), (1, 3, 2)):
            Xs = [x[:, :c].contiguous() for x, c in zip(Xw, widths)]
            Outs = [torch.empty_like(x) for x in Xs]
            hb.hbs_apply_batch(h, Xs, Outs, trans=trans)
            for j, (o, c) in enumerate(zip(Outs, widths)):
                assert torch.equal(o, wide[j][:, :c]), (trans, widths, j)


def test_blackbox_callback_pipeline(hb):
    # sampling through a callback that applies the generator handle (Section 1 black box)
    N, k, r, s, leaf, seed = 1000, 6, 9, 27, 18, 21
    g = exact_hbs(N, leaf, k, 2)
    A = g.dense()
    gen = generator_handle(hb, [g], [leaf])

    def op(trans, X, Out):
        hb.hbs_apply(gen, X, Out, trans=bool(trans))

    Om, Ps, Y, Z = zeros(N, s)
    hb.hbs_sample(op, s, seed, Om, Ps, Y, Z, N=N)
    h = hb.hbs_compress([hb.Problem(N, r, s, leaf, Om, Ps, Y, Z)])
    X = torch.eye(N, dtype=torch.float64, device="cuda")
    Out = torch.empty_like(X)
    hb.hbs_apply(h, X, Out)
    hb.hbs_sync_status(h)
    At = Out.cpu().numpy()
    assert rel(At, A) <= 1e-11
    Ao = oapply.dense(ocompress(*osample(lambda x, t: (A.T if t else A) @ x, N, s, seed), r, leaf))
    assert rel(At, Ao) <= 1e-10


def test_callback_error_is_reported(hb):
    N, s = 64, 12

    def op(trans, X, Out):
        raise RuntimeError("operator failed")

    with pytest.raises(hb.HBSError) as e:
        hb.hbs_sample(op, s, 1, *zeros(N, s), N=N)
    assert e.value.code == -7


def test_batched_blackbox_compression(hb):
    # several exact-HBS operators of different N and k sampled by one batched apply and
    # compressed by one launch per tree height
    shapes = [(1000, 6), (512, 8), (1024, 5), (2048, 10), (256, 4), (1024, 7)]
    gens, leafs = [], []
    for j, (N, k) in enumerate(shapes):
        leaf = 1 << int(np.floor(np.log2(2 * k)))
        gens.append(exact_hbs(N, leaf, k, 40 + j))
        leafs.append(leaf)
    gen = generator_handle(hb, gens, leafs)
    Oms, Pss, Ys, Zs, probs = [], [], [], [], []
    for j, (g, leaf) in enumerate(zip(gens, leafs)):
        r = min(g.k + 2, min(g.sizes[2 ** g.L: 2 ** (g.L + 1)]))      # r = k + p, at most a leaf
        s = 3 * r
        Om, Ps, Y, Z = zeros(g.N, s)
        hb.hbs_draw_gaussian(g.N, s, 0, 100 + j, Om)
        hb.hbs_draw_gaussian(g.N, s, 1, 100 + j, Ps)
        Oms.append(Om), Pss.append(Ps), Ys.append(Y), Zs.append(Z)
        probs.append(hb.Problem(g.N, r, s, leaf, Om, Ps, Y, Z))
    hb.hbs_apply_batch(gen, Oms, Ys)
    hb.hbs_apply_batch(gen, Pss, Zs, trans=True)
    for j, g in enumerate(gens):                       # batched apply = per-item apply
        ref = torch.empty_like(Ys[j])
        hb.hbs_apply(gen, Oms[j], ref, item=j)
        torch.cuda.synchronize()
        assert torch.equal(ref, Ys[j])
    h = hb.hbs_compress(probs)
    hb.hbs_sync_status(h)
    for j, g in enumerate(gens):
        X = torch.eye(g.N, dtype=torch.float64, device="cuda")
        Out = torch.empty_like(X)
        hb.hbs_apply(h, X, Out, item=j)
        torch.cuda.synchronize()
        assert rel(Out.cpu().numpy(), g.dense()) <= 1e-11, j


def test_graph_replay_and_tuning_change_nothing(hb):
    N, r, s, leaf = 2048, 40, 120, 64
    x = [torch.as_tensor(gaussian((N, s), 60 + i), device="cuda") for i in range(4)]
    prob = hb.Problem(N, r, s, leaf, *x)
    h = hb.hbs_plan([prob])

    def factors():
        hb.hbs_sync_status(h)
        return [hb.hbs_get_node(h, t)[2] for t in (1, 2, 17, 40, 63)]

    hb.hbs_execute(h, [prob])                          # captures the graph
    ref = factors()
    hb.hbs_execute(h, [prob])                          # replays it
    for a, b in zip(ref, factors()):
        assert torch.equal(a, b)
    hb.hbs_set_graph(h, False)
    hb.hbs_execute(h, [prob])                          # plain launches
    for a, b in zip(ref, factors()):
        assert torch.equal(a, b)
    hb.hbs_set_graph(h, True)
    hb.hbs_autotune(h)
    R = hb.hbs_get_tuning(h)
    assert len(R) == 6 and all(v != 0 and -8 <= v <= 16 for v in R)
    hb.hbs_execute(h, [prob])                          # row slicing never changes the arithmetic
    for a, b in zip(ref, factors()):
        assert torch.equal(a, b)
    # row slices (R > 0) and clusters sharing one factorization (R = -C, C rows owners) round
    # exactly alike, whatever the split: C = 3 leaves ragged row ownership at n = 64 and 80
    for tuning in ([1] * len(R), [-1] * len(R), [-2] * len(R), [-3] * len(R), [-8] * len(R),
                   [-5, 3, -7, 2, -4, -6]):
        hb.hbs_set_tuning(h, tuning)
        assert hb.hbs_get_tuning(h) == tuning
        hb.hbs_execute(h, [prob])
        for a, b in zip(ref, factors()):
            assert torch.equal(a, b)

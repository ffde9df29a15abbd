"""Batched MPK (one plan and one launch for several matrices) against the oracle, block by
block, bit for bit; alone and in the batch the results are the same."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_12525_gb300 as m
    m.build()
    m.load()
    return m


def _disconnected():
    n = 9
    e = [(0, 1), (1, 2), (3, 4), (6, 7)]
    r = list(range(n)) + [u for u, v in e] + [v for u, v in e]
    c = list(range(n)) + [v for u, v in e] + [u for u, v in e]
    return gen.from_coo(n, r, c, np.linspace(-1, 1, len(r)))


def _blocks():
    return [
        (gen.laplacian_3d(9, 8, 7), True, 5),
        (gen.stencil27(6), True, 3),
        (gen.banded_random(800, stream=501), True, 8),
        (gen.xxz_chain(8, stream=502), True, 6),
        (_disconnected(), False, 4),
        (gen.CSR([0, 1], [0], np.array([2.0])), True, 2),
        (gen.laplacian_2d(30, 20), True, 7),
    ]


def _bits_equal(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("m", [1, 2])
def test_batch_bit_exact_per_block(mpk, order, m):
    blocks = _blocks()
    mats = [mpk.CsrMatrix.from_host(A, is_symmetric=sym) for A, sym, _ in blocks]
    p_each = [p for _, _, p in blocks]
    B = mpk.batch_plan(mats, p_each, p_max=8, nrhs=m, cache_bytes=30000, chunk_rows=64, order=order)
    d = B.describe()
    assert d["count"] == len(blocks) and d["powers"] == p_each
    offs = np.cumsum([0] + [A.n for A, _, _ in blocks]).tolist()
    assert d["row_offsets"] == offs
    # groups never span two blocks
    assert set(offs) <= set(B.group_row_ptr.cpu().numpy().tolist())
    Xs, want = [], []
    for i, (A, _, p) in enumerate(blocks):
        X = gen.vector(A.n, m, stream=510 + i)
        Yo = oracle.mpk(A, X, p)
        if order == mpk.ORDER_PLAN:
            pe = oracle.levels(A, 0)[1]
            X, Yo = np.ascontiguousarray(X[pe]), np.ascontiguousarray(Yo[:, pe, :])
        Xs.append(torch.from_numpy(X).cuda())
        want.append(Yo)
    Ys = [torch.full((p + 1, A.n, m), float("nan"), dtype=torch.float64, device="cuda") for A, _, p in blocks]
    B.apply(Xs, Ys)
    torch.cuda.synchronize()
    for Y, Yo in zip(Ys, want):
        assert _bits_equal(Y.cpu().numpy(), Yo)


def test_batch_equals_blocks_alone(mpk):
    blocks = _blocks()
    mats = [mpk.CsrMatrix.from_host(A, is_symmetric=sym) for A, sym, _ in blocks]
    p_each = [p for _, _, p in blocks]
    B = mpk.batch_plan(mats, p_each, nrhs=1)
    Xs = [torch.from_numpy(gen.vector(A.n, 1, stream=520 + i)).cuda() for i, (A, _, _) in enumerate(blocks)]
    Ys = B.apply(Xs)
    for (A, sym, p), dA, X, Y in zip(blocks, mats, Xs, Ys):
        P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=p)
        Ya = P.apply(X, p)
        P.sync_status()
        assert torch.equal(Ya, Y)


def test_batch_narrow_values_and_graph_replay(mpk):
    # bfloat16 stencil blocks (exact coefficients), replayed from a CUDA graph
    blocks = [gen.stencil27(7), gen.laplacian_3d(10, 9, 8), gen.stencil27(5)]
    mats = [mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16) for A in blocks]
    p_each = [4, 6, 2]
    B = mpk.batch_plan(mats, p_each, nrhs=2, cache_bytes=50000)
    Xs = [torch.zeros((A.n, 2), dtype=torch.float64, device="cuda") for A in blocks]
    Ys = [torch.zeros((p + 1, A.n, 2), dtype=torch.float64, device="cuda") for A, p in zip(blocks, p_each)]
    B.apply(Xs, Ys)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.apply(Xs, Ys)
    for seed in (530, 531):
        host = [gen.vector(A.n, 2, stream=seed + i) for i, A in enumerate(blocks)]
        for X, h in zip(Xs, host):
            X.copy_(torch.from_numpy(h))
        g.replay()
        torch.cuda.synchronize()
        for A, h, Y, p in zip(blocks, host, Ys, p_each):
            assert _bits_equal(Y.cpu().numpy(), oracle.mpk(A, h, p))


def test_batch_rejects_mixed_types_and_single_plan_calls(mpk):
    A = gen.laplacian_2d(10, 10)
    a64 = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    a32 = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_F32)
    with pytest.raises(mpk.MpkError):
        mpk.batch_plan([a64, a32], [2, 2])
    with pytest.raises(mpk.MpkError):
        mpk.batch_plan([a64], [9], p_max=8)
    B = mpk.batch_plan([a64, a64], [2, 3])
    X = torch.zeros((A.n, 1), dtype=torch.float64, device="cuda")
    Y = torch.zeros((3, A.n, 1), dtype=torch.float64, device="cuda")
    assert B._lib.mpk_apply(B._h, X.data_ptr(), 2, Y.data_ptr(), None) == mpk.MPK_ERR_INVALID


def test_batch_in_place_views(mpk):
    blocks = _blocks()
    mats = [mpk.CsrMatrix.from_host(A, is_symmetric=sym) for A, sym, _ in blocks]
    p_each = [p for _, _, p in blocks]
    B = mpk.batch_plan(mats, p_each, nrhs=2, order=mpk.ORDER_PLAN)
    host = [gen.vector(A.n, 2, stream=540 + i) for i, (A, _, _) in enumerate(blocks)]
    perms = [oracle.levels(A, 0)[1] for A, _, _ in blocks]
    Xs = [torch.from_numpy(np.ascontiguousarray(h[pe])).cuda() for h, pe in zip(host, perms)]
    views = B.apply(Xs, in_place=True)
    torch.cuda.synchronize()
    for (A, _, p), h, pe, V in zip(blocks, host, perms, views):
        assert _bits_equal(V.cpu().numpy(), oracle.mpk(A, h, p)[:, pe, :])

"""Full-size parity on the 256^3 7-point Laplacian (n = 16,777,216, nnz = 117,047,296), p = 8.

The headline case runs exactly as bench.py times it: plan order (X and Y in the BFS
numbering), the default cache budget, the automatically chosen block shape with its default
chunk rows, one kernel launch.  The other cases run the original row order (gather, kernel,
permuted write) on the staged and the warp-ticketed engine, bulky levels split, and binary32
accumulation against the oracle's binary32 path.  Levels, permutation and every one of the
8 x 16.7M output values are compared with the oracle bit for bit."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A, p = gen.config_headline(256)
    X = gen.vector(A.n, 1, stream=1)
    return A, X, p, oracle.mpk(A, X, p)


@pytest.fixture(scope="module")
def levels(workload):
    import paper_2405_12525_gb300 as mpk
    mpk.build()
    A, X, p, want = workload
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    return mpk, dA, L


def _check(Yg, want):
    assert np.array_equal(Yg.view(np.uint64), want.view(np.uint64))
    for k in range(1, want.shape[0]):
        assert np.linalg.norm(Yg[k] - want[k]) / np.linalg.norm(want[k]) <= 1e-13


def test_headline_levels_bit_exact(workload, levels):
    A, X, p, want = workload
    mpk, dA, L = levels
    assert L.num_levels == 766
    level_of = L.level_of.cpu().numpy()
    i = np.arange(A.n)
    assert np.array_equal(level_of, i % 256 + (i // 256) % 256 + i // 65536)
    _, pe, _, lp = oracle.levels(A, 0)
    assert np.array_equal(L.perm.cpu().numpy(), pe)
    assert np.array_equal(L.level_ptr.cpu().numpy(), lp)


def test_headline_bench_configuration_bit_exact(workload, levels):
    # bench.py's headline: mpk.plan(dA, L, p_max=8, nrhs=1, order=ORDER_PLAN) with every other
    # option at its default, X permuted into plan order, one apply into Y
    A, X, p, want = workload
    mpk, dA, L = levels
    P = mpk.plan(dA, L, p_max=p, nrhs=1, order=mpk.ORDER_PLAN)
    d = P.describe()
    assert d["shape"] == 1 and d["chunk_rows"] == 512 and d["split_levels"] == 0 and d["accum"] == 0
    perm = L.perm.long()
    Xp = torch.from_numpy(X).cuda()[perm].contiguous()
    Y = torch.full((p + 1, A.n, 1), float("nan"), dtype=torch.float64, device="cuda")
    P.apply(Xp, p, Y=Y)
    P.sync_status()
    Yg = Y.cpu().numpy()
    del Y
    _check(Yg, want[:, perm.cpu().numpy(), :])


@pytest.mark.parametrize("engine,split", [(0, False), (1, False), (0, True)])
def test_headline_original_order_bit_exact(workload, levels, engine, split):
    A, X, p, want = workload
    mpk, dA, L = levels
    P = mpk.plan(dA, L, p_max=p, nrhs=1, order=mpk.ORDER_ORIGINAL, engine=engine, split_levels=split)
    Y = torch.full((p + 1, A.n, 1), float("nan"), dtype=torch.float64, device="cuda")
    P.apply(torch.from_numpy(X).cuda(), p, Y=Y)
    P.sync_status()
    Yg = Y.cpu().numpy()
    del Y
    _check(Yg, want)


def test_headline_binary32_accumulation_bit_exact(workload):
    # bench.py --accum f32: bfloat16 values ({6, -1} exact), binary32 row sums, plan order
    import paper_2405_12525_gb300 as mpk
    mpk.build()
    A, X, p, _ = workload
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=p, nrhs=1, order=mpk.ORDER_PLAN, accum=mpk.MPK_F32)
    perm = L.perm.long()
    Xp = torch.from_numpy(X).cuda()[perm].contiguous()
    Y = torch.full((p + 1, A.n, 1), float("nan"), dtype=torch.float64, device="cuda")
    P.apply(Xp, p, Y=Y)
    P.sync_status()
    Yg = Y.cpu().numpy()
    del Y
    want = oracle.mpk_acc32(A, X, p)[:, perm.cpu().numpy(), :]
    assert np.array_equal(Yg.view(np.uint64), want.view(np.uint64))

"""Full-size parity on the 256^3 7-point Laplacian (n = 16,777,216, nnz = 117,047,296), p = 8,
in the launch configuration bench.py times (default cache budget, 512-row chunks, original
row order), on both engines of the level-blocked kernel.  Levels, permutation and every one
of the 8 x 16.7M output values are compared with the oracle bit for bit."""
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


@pytest.mark.parametrize("engine", [0, 1])
def test_headline_levels_and_powers_bit_exact(workload, engine):
    import paper_2405_12525_gb300 as mpk
    mpk.build()
    A, X, p, want = workload
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    assert L.num_levels == 766
    level_of = L.level_of.cpu().numpy()
    i = np.arange(A.n)
    assert np.array_equal(level_of, i % 256 + (i // 256) % 256 + i // 65536)
    _, pe, _, lp = oracle.levels(A, 0)
    assert np.array_equal(L.perm.cpu().numpy(), pe)
    assert np.array_equal(L.level_ptr.cpu().numpy(), lp)
    P = mpk.plan(dA, L, p_max=p, nrhs=1, order=mpk.ORDER_ORIGINAL, engine=engine)
    Y = torch.full((p + 1, A.n, 1), float("nan"), dtype=torch.float64, device="cuda")
    P.apply(torch.from_numpy(X).cuda(), p, Y=Y)
    P.sync_status()
    Yg = Y.cpu().numpy()
    del Y
    assert np.array_equal(Yg.view(np.uint64), want.view(np.uint64))
    for k in range(1, p + 1):
        assert np.linalg.norm(Yg[k] - want[k]) / np.linalg.norm(want[k]) <= 1e-13

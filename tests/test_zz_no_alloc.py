"""mpk_apply_noalloc: the level-blocked MPK for callers that cannot allocate device memory
during a call (e.g. while their allocator is locked, or in loops that must not pay the
implicit synchronisation of cudaMalloc/cudaFree).  Its synchronisation state lives in a
fixed array inside the library; the results must match mpk_apply's."""
import numpy as np
import pytest

import gen

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


def test_noalloc_matches_apply_on_two_calls_in_a_row(mpk):
    A = gen.laplacian_3d(40, 33, 21)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=8, nrhs=1, order=mpk.ORDER_PLAN, cache_bytes=400000)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call, (stream_id, p) in enumerate([(11, 8), (12, 5)]):
        X = torch.from_numpy(gen.vector(A.n, 1, stream=stream_id)).cuda()
        want = P.apply(X, p)
        P.sync_status()
        Y = torch.full((p + 1, A.n, 1), float("nan"), dtype=torch.float64, device="cuda")
        P.apply_noalloc(X, p, Y, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"call {call}: status {int(status.item())}"
        # same arithmetic as mpk_apply: identical bits, and within the FP64 tolerance of 1e-13
        assert torch.equal(Y, want), f"call {call}"
        for k in range(1, p + 1):
            assert (torch.linalg.norm(Y[k] - want[k]) / torch.linalg.norm(want[k])).item() <= 1e-13


def test_noalloc_rejects_too_many_chunks_and_original_order(mpk):
    A = gen.laplacian_3d(128, 128, 64)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    # 1,048,576 rows in 32-row chunks: 32,768+ chunks x 32 powers exceeds the 2^20-word scratch
    P = mpk.plan(dA, L, p_max=31, nrhs=1, order=mpk.ORDER_PLAN, chunk_rows=32)
    X = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    Y = torch.empty((32, A.n, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(mpk.MpkError) as e:
        P.apply_noalloc(X, 31, Y)
    assert e.value.status == 2
    Po = mpk.plan(dA, L, p_max=2, nrhs=1, order=mpk.ORDER_ORIGINAL)
    with pytest.raises(mpk.MpkError) as e:
        Po.apply_noalloc(X, 2, torch.empty((3, A.n, 1), dtype=torch.float64, device="cuda"))
    assert e.value.status == 7


def test_noalloc_p0_and_checked_outputs(mpk):
    # p = 0 copies X into Y[0], as mpk_apply does; outputs too small for the call, or a status
    # word that is not a device int32, are refused before anything reaches the GPU
    A = gen.laplacian_3d(12, 10, 8)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=4, nrhs=1, order=mpk.ORDER_PLAN)
    X = torch.from_numpy(gen.vector(A.n, 1, stream=13)).cuda()
    Y = torch.full((1, A.n, 1), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    P.apply_noalloc(X, 0, Y, status=status)
    torch.cuda.synchronize()
    assert torch.equal(Y[0], X.view(A.n, 1)) and int(status.item()) == 0
    with pytest.raises(ValueError):
        P.apply_noalloc(X, 3, torch.empty((3, A.n, 1), dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        P.apply_noalloc(X, 1, torch.empty((2, A.n, 1), dtype=torch.float64, device="cuda"),
                        status=torch.zeros(1, dtype=torch.int64, device="cuda"))
    with pytest.raises(TypeError):
        P.apply_noalloc(X, 1, torch.empty((2, A.n, 1), dtype=torch.float32, device="cuda"))


def test_noalloc_leaves_device_memory_unchanged(mpk):
    # after one warm-up call (lazy module loading, the scratch address lookup), further calls
    # take no device memory: the free bytes the driver reports stay the same
    A = gen.laplacian_3d(48, 40, 32)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=8, nrhs=1, order=mpk.ORDER_PLAN)
    X = torch.from_numpy(gen.vector(A.n, 1, stream=31)).cuda()
    Y = torch.empty((9, A.n, 1), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    P.apply_noalloc(X, 8, Y, status=status)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for p in (8, 3, 0, 8):
        P.apply_noalloc(X, p, Y, status=status)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert int(status.item()) == 0
    assert free1 == free0

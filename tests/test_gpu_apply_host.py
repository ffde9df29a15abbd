"""mpk_apply_host: the powers of Sec. 3 with X and Y in host memory.  The results equal the
oracle and mpk_apply bit for bit in both orders, on every engine, with binary32 row sums
(including the two-slice block shape), for level-capped plans, p = 0 and p < p_max; pageable or
overlapping outputs are refused before any work is queued."""
import ctypes

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


def _bits(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint64), np.ascontiguousarray(b).view(np.uint64))


def _pinned_nan(shape):
    return torch.full(shape, float("nan"), dtype=torch.float64).pin_memory()


@pytest.mark.parametrize("pin", [False, True])
@pytest.mark.parametrize("engine", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_host_buffers_equal_oracle_and_device_apply(mpk, order, m, engine, pin):
    A = gen.laplacian_3d(21, 13, 11)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=7, nrhs=m, order=order, cache_bytes=60000, engine=engine)
    _, pe, _, _ = oracle.levels(A, 0)
    X = gen.vector(A.n, m, stream=501)
    Xin = np.ascontiguousarray(X if order == 0 else X[pe])
    Xh = torch.from_numpy(Xin).pin_memory() if pin else torch.from_numpy(Xin)
    Yh = _pinned_nan((8, A.n, m))
    P.apply_host(Xh, 7, Yh)
    torch.cuda.synchronize()
    P.sync_status()
    want = oracle.mpk(A, X, 7)
    assert _bits(Yh.numpy(), want if order == 0 else want[:, pe, :])
    Yd = P.apply(torch.from_numpy(Xin).cuda(), 7)
    P.sync_status()
    assert _bits(Yd.cpu().numpy(), Yh.numpy())


@pytest.mark.parametrize("shape", [0, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_host_buffers_binary32(mpk, order, shape):
    # plan option shape 0: the planner's choice (two slices a warp, index 4); 2: index 1
    A = gen.laplacian_3d(40, 36, 30)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    Aw = gen.CSR(dA.row_ptr.cpu().numpy(), dA.col.cpu().numpy(), dA.val.double().cpu().numpy())
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=8, order=order, accum=mpk.MPK_F32, shape=shape)
    assert P.describe()["shape"] == (4 if shape == 0 else 1)
    _, pe, _, _ = oracle.levels(A, 0)
    X = gen.vector(A.n, 1, stream=502)
    Xin = np.ascontiguousarray(X if order == 0 else X[pe])
    Yh = P.apply_host(torch.from_numpy(Xin).pin_memory(), 8, _pinned_nan((9, A.n, 1)))
    torch.cuda.synchronize()
    P.sync_status()
    want = oracle.mpk_acc32(Aw, X, 8)
    assert _bits(Yh.numpy(), want if order == 0 else want[:, pe, :])


@pytest.mark.parametrize("order", [0, 1])
def test_host_buffers_x_staged_shape(mpk, order):
    # the shape that stages input rows with bulk copies (plan option 4) through the host-output mode
    A = gen.laplacian_3d(21, 13, 11)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=6, order=order, cache_bytes=60000, shape=4)
    assert P.describe()["shape"] == 3
    _, pe, _, _ = oracle.levels(A, 0)
    X = gen.vector(A.n, 1, stream=507)
    Xin = np.ascontiguousarray(X if order == 0 else X[pe])
    Yh = P.apply_host(torch.from_numpy(Xin).pin_memory(), 6, _pinned_nan((7, A.n, 1)))
    torch.cuda.synchronize()
    P.sync_status()
    want = oracle.mpk(A, X, 6)
    assert _bits(Yh.numpy(), want if order == 0 else want[:, pe, :])


def test_host_buffers_level_capped_plan(mpk):
    # level 0 has no units: its rows of Y[0] are copied on the host side of the call
    A = gen.laplacian_3d(17, 9, 6)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=5, order=mpk.ORDER_PLAN, level_capped=True)
    X = torch.from_numpy(gen.vector(A.n, 1, stream=503))
    Yd = P.apply(X.cuda(), 5, Y=torch.full((6, A.n, 1), float("nan"), dtype=torch.float64, device="cuda"))
    Yh = P.apply_host(X, 5, _pinned_nan((6, A.n, 1)))
    torch.cuda.synchronize()
    P.sync_status()
    assert _bits(Yd.cpu().numpy(), Yh.numpy())


@pytest.mark.parametrize("order", [0, 1])
def test_host_buffers_small_p(mpk, order):
    A = gen.banded_random(3000, stream=504)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=7, order=order, cache_bytes=40000)
    _, pe, _, _ = oracle.levels(A, 0)
    X = gen.vector(A.n, 1, stream=505)
    Xin = np.ascontiguousarray(X if order == 0 else X[pe])
    want = oracle.mpk(A, X, 3)
    want = want if order == 0 else want[:, pe, :]
    for p in (0, 1, 3):
        Yh = P.apply_host(torch.from_numpy(Xin), p, _pinned_nan((p + 1, A.n, 1)))
        torch.cuda.synchronize()
        P.sync_status()
        assert _bits(Yh.numpy(), want[: p + 1])


def test_host_buffers_refused(mpk):
    A = gen.laplacian_2d(20, 20)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=4, order=mpk.ORDER_PLAN)
    X = torch.from_numpy(gen.vector(A.n, 1, stream=506))
    with pytest.raises(TypeError):  # the binding wants a pinned output
        P.apply_host(X, 3, torch.empty((4, A.n, 1), dtype=torch.float64))
    # the library checks on its own: a pageable output is refused with MPK_ERR_INVALID
    Yp = np.empty((4, A.n, 1))
    st = P._lib.mpk_apply_host(P._h, X.data_ptr(), 3, Yp.ctypes.data_as(ctypes.c_void_p),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 1
    # an output that overlaps the input
    Yh = _pinned_nan((4, A.n, 1))
    with pytest.raises(mpk.MpkError) as e:
        P.apply_host(Yh[1], 3, Yh)
    assert e.value.status == 1
    torch.cuda.synchronize()
    P.sync_status()

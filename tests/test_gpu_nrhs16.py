"""Blocks of 16 right-hand sides in one plan: the unstaged block shape (one block per SM, a
row's 16 x values and sums in registers) and the sweep engine, bit for bit against the oracle
in both orders, for powers, the comparator, the Chebyshev filter (real and complex) and binary32
row sums; the staged shapes and the warp engine refuse 16 columns."""
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


MATS = {
    "lap3d_17x9x6": (lambda: gen.laplacian_3d(17, 9, 6), True),
    "band_3000": (lambda: gen.banded_random(3000, stream=171), True),
    "int_nonsym_500": (lambda: gen.random_int_matrix(500, 5, stream=172), False),
    "xxz_10": (lambda: gen.xxz_chain(10, stream=173), True),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("engine", [0, 2])
def test_powers_16_columns_bit_exact(mpk, name, order, engine):
    make, sym = MATS[name]
    A = make()
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=sym)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=7, nrhs=16, order=order, cache_bytes=60000, engine=engine)
    d = P.describe()
    assert d["nrhs"] == 16 and d["shape"] == 2
    X = gen.vector(A.n, 16, stream=174)
    _, pe, _, _ = oracle.levels(A, 0)
    want = oracle.mpk(A, X, 7)
    Xin = X if order == 0 else np.ascontiguousarray(X[pe])
    Y = torch.full((8, A.n, 16), float("nan"), dtype=torch.float64, device="cuda")
    P.apply(torch.from_numpy(Xin).cuda(), 7, Y=Y)
    P.sync_status()
    got = Y.cpu().numpy()
    assert _bits(got, want if order == 0 else want[:, pe, :])
    # the comparator (p separate SpMV launches) gives the same bits
    Y2 = torch.full((8, A.n, 16), float("nan"), dtype=torch.float64, device="cuda")
    P.spmv_powers(torch.from_numpy(Xin).cuda(), 7, Y=Y2)
    assert torch.equal(Y2, Y)


def test_chebyshev_16_columns_real_and_complex(mpk):
    A = gen.laplacian_3d(12, 10, 9)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    lo, hi = gen.gershgorin_bounds(A)
    a, c = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, nrhs=16, cache_bytes=40000)
    X = gen.vector(A.n, 16, stream=175)
    deg = 19
    cr = gen.uniform(gen.derive_seed(176), deg + 1)
    ci = gen.uniform(gen.derive_seed(177), deg + 1)
    got = P.cheb_filter(torch.from_numpy(X).cuda(), deg, cr, scale=a, shift=c).cpu().numpy()
    P.sync_status()
    assert _bits(got, oracle.cheb(A, X, deg, cr, scale=a, shift=c))
    got = P.cheb_filter(torch.from_numpy(X).cuda(), deg, cr, ci, scale=a, shift=c).cpu().numpy()
    P.sync_status()
    assert _bits(got, oracle.cheb(A, X, deg, cr, ci, scale=a, shift=c))


def test_binary32_sums_16_columns(mpk):
    A = gen.laplacian_3d(15, 11, 8)  # {6, -1}: exact in bfloat16
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    L = mpk.build_levels(dA, 0)
    _, pe, _, _ = oracle.levels(A, 0)
    X = gen.vector(A.n, 16, stream=178)
    want = oracle.mpk_acc32(A, X, 6)
    for engine in (0, 2):
        P = mpk.plan(dA, L, p_max=6, nrhs=16, order=mpk.ORDER_PLAN, accum=mpk.MPK_F32, engine=engine)
        Y = torch.full((7, A.n, 16), float("nan"), dtype=torch.float64, device="cuda")
        P.apply(torch.from_numpy(np.ascontiguousarray(X[pe])).cuda(), 6, Y=Y)
        P.sync_status()
        assert _bits(Y.cpu().numpy(), want[:, pe, :])


def test_16_columns_refuse_staged_shapes_and_the_warp_engine(mpk):
    A = gen.laplacian_3d(9, 8, 7)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    for kwargs in ({"shape": 1}, {"shape": 2}, {"shape": 4}, {"engine": 1}):
        with pytest.raises(mpk.MpkError) as e:
            mpk.plan(dA, L, p_max=4, nrhs=16, **kwargs)
        assert e.value.status == 7  # MPK_ERR_UNSUPPORTED
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, L, p_max=4, nrhs=12)

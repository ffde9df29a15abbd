"""Binary32 accumulation (the precision option): values stored as float32 or bfloat16, each
row sum in binary32 over the binary32 rounding of its input, vectors and the Chebyshev
recurrence in binary64.

The oracle's binary32 path (oracle.mpk_acc32 / oracle.cheb_acc32, on torch's widening of the
stored values) defines the results bit for bit, for the level-blocked engine (every block
shape that takes the option) and the unblocked sweep.  The error against the binary64
oracle is stated for every power and bounded.
"""
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


def _widened(dA):
    return gen.CSR(dA.row_ptr.cpu().numpy(), dA.col.cpu().numpy(), dA.val.double().cpu().numpy())


def _poisoned(shape):
    return torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")


def _bits_equal(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


MATS = {
    "lap3d_21x13x11": lambda: gen.laplacian_3d(21, 13, 11),
    "lap2d_64": lambda: gen.laplacian_2d(64, 64),
    "band_3000": lambda: gen.banded_random(3000, stream=71),
    "xxz_10": lambda: gen.xxz_chain(10, stream=73),
    "stencil27_9": lambda: gen.stencil27(9),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("vtype", ["f32", "bf16"])
@pytest.mark.parametrize("engine,shape", [(0, 0), (0, 1), (0, 2), (0, 3), (0, 5), (2, 0)])
def test_powers_bit_exact(mpk, name, vtype, engine, shape):
    A = MATS[name]()
    vt = {"f32": mpk.MPK_F32, "bf16": mpk.MPK_BF16}[vtype]
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vt)
    Aw = _widened(dA)
    L = mpk.build_levels(dA, 0)
    pe = L.perm.cpu().numpy()
    X = gen.vector(A.n, 2, stream=401)
    Yo = oracle.mpk_acc32(Aw, X, 7)
    for order in (0, 1):
        P = mpk.plan(dA, L, p_max=7, nrhs=2, cache_bytes=50000, order=order, engine=engine, shape=shape,
                     accum=mpk.MPK_F32)
        assert P.describe()["accum"] == mpk.MPK_F32
        Xin = X if order == 0 else np.ascontiguousarray(X[pe])
        for p in (1, 4, 7):
            Y = P.apply(torch.from_numpy(Xin).cuda(), p, Y=_poisoned((p + 1, A.n, 2)))
            P.sync_status()
            want = Yo[: p + 1] if order == 0 else Yo[: p + 1][:, pe, :]
            assert _bits_equal(Y.cpu().numpy(), want), (order, p)


@pytest.mark.parametrize("m", [1, 2, 4, 8])
@pytest.mark.parametrize("chunk_rows", [32, 416])
def test_powers_nrhs_and_chunks(mpk, m, chunk_rows):
    A = gen.laplacian_3d(19, 11, 7)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_F32)
    L = mpk.build_levels(dA, 0)
    pe = L.perm.cpu().numpy()
    X = gen.vector(A.n, m, stream=402)
    P = mpk.plan(dA, L, p_max=8, nrhs=m, cache_bytes=200000, chunk_rows=chunk_rows, order=mpk.ORDER_PLAN,
                 accum=mpk.MPK_F32)
    Y = P.apply(torch.from_numpy(np.ascontiguousarray(X[pe])).cuda(), 8, Y=_poisoned((9, A.n, m)))
    P.sync_status()
    assert _bits_equal(Y.cpu().numpy(), oracle.mpk_acc32(_widened(dA), X, 8)[:, pe, :])


def test_error_against_binary64_per_power(mpk):
    # 3-D Laplacian {6, -1} (exact in bfloat16), x ~ U[-1, 1): the only error is binary32
    # accumulation; stated per power and bounded.  Each power adds at most gamma_7 = 7 u of the
    # row's absolute sum (u = 2^-24), on top of the propagated error of its input; with
    # ||A||_inf = 12 the propagated error grows at most like sum_k 12^k / ||A^k x||, so the test
    # takes the bound 2 * 7 u * k * (12^k ||x|| / ||A^k x||) for power k.
    A = gen.laplacian_3d(24, 20, 16)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    L = mpk.build_levels(dA, 0)
    X = gen.vector(A.n, 1, stream=403)
    P = mpk.plan(dA, L, p_max=8, accum=mpk.MPK_F32)
    Y = P.apply(torch.from_numpy(X).cuda(), 8).cpu().numpy()
    P.sync_status()
    Y64 = oracle.mpk(A, X, 8)
    u = 2.0 ** -24
    errs = []
    for k in range(1, 9):
        rel = np.linalg.norm(Y[k] - Y64[k]) / np.linalg.norm(Y64[k])
        errs.append(rel)
        bound = 2 * 7 * u * k * (12.0 ** k * np.linalg.norm(X) / np.linalg.norm(Y64[k]))
        assert 0 < rel <= bound, (k, rel, bound)
    print("\nbinary32 accumulation, 3-D Laplacian 24x20x16, relative error per power 1..8 = "
          + ", ".join(f"{e:.2e}" for e in errs))


@pytest.mark.parametrize("engine", [0, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_chebyshev_bit_exact_and_resumable(mpk, engine, order):
    A = gen.xxz_chain(12, stream=87)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_F32)
    Aw = _widened(dA)
    lo, hi = gen.gershgorin_bounds(A)
    scale, shift = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    L = mpk.build_levels(dA, 0)
    _, pe, ip, _ = oracle.levels(A, 0)
    P = mpk.plan(dA, L, p_max=8, nrhs=2, order=order, cache_bytes=30000, engine=engine, accum=mpk.MPK_F32)
    X = gen.vector(A.n, 2, stream=404)
    Xin = torch.from_numpy(np.ascontiguousarray(X if order == 0 else X[pe])).cuda()
    deg = 29
    cr = gen.uniform(gen.derive_seed(405), deg + 1)
    ci = gen.uniform(gen.derive_seed(406), deg + 1)
    whole = P.cheb_filter(Xin, deg, cr, ci, scale=scale, shift=shift).cpu().numpy()
    P.sync_status()
    want = oracle.cheb_acc32(Aw, X, deg, cr, ci, scale=scale, shift=shift)
    got = whole[ip] if order == 1 else whole
    assert _bits_equal(got, want)
    # pieces and a host checkpoint give the same bits (the binary32 input is rebuilt from the state)
    st = P.cheb_state()
    P.cheb_begin(Xin, st, cr[0], ci[0])
    P.cheb_advance(st, 0, 11, cr, ci, scale=scale, shift=shift)
    saved = st.cpu().numpy().copy()
    st.copy_(torch.from_numpy(saved))
    P.cheb_advance(st, 11, deg, cr, ci, scale=scale, shift=shift)
    assert _bits_equal(P.cheb_finish(st).cpu().numpy(), whole)
    # real coefficients too
    wr = P.cheb_filter(Xin, 13, cr, scale=scale, shift=shift).cpu().numpy()
    wr = wr[ip] if order == 1 else wr
    assert _bits_equal(wr, oracle.cheb_acc32(Aw, X, 13, cr, scale=scale, shift=shift))


def test_no_allocation_entry_point_accum32(mpk):
    A = gen.laplacian_3d(21, 13, 11)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=6, order=mpk.ORDER_PLAN, accum=mpk.MPK_F32)
    X = torch.from_numpy(gen.vector(A.n, 1, stream=407)).cuda()
    Ya = P.apply(X, 6)
    Yn = P.apply_noalloc(X, 6, _poisoned((7, A.n, 1)))
    P.sync_status()
    assert torch.equal(Ya, Yn)


def test_rejected_combinations(mpk):
    A = gen.laplacian_2d(16, 16)
    d64 = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    d32 = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_F32)
    L = mpk.build_levels(d32, 0)
    for kwargs in ({"dA": d64}, {"engine": 1}, {"trace": True}, {"shape": 4}, {"accum": 5}):
        dA = kwargs.pop("dA", d32)
        acc = kwargs.pop("accum", mpk.MPK_F32)
        with pytest.raises(mpk.MpkError) as e:
            mpk.plan(dA, L, p_max=3, accum=acc, **kwargs)
        assert e.value.status in (1, 7)
    P = mpk.plan(d32, L, p_max=3, accum=mpk.MPK_F32)
    with pytest.raises(mpk.MpkError) as e:
        P.spmv_powers(torch.zeros((A.n, 1), dtype=torch.float64, device="cuda"), 2)
    assert e.value.status == 7


def test_automatic_two_slice_shape_for_bfloat16(mpk):
    # binary32 sums over bfloat16 values, one right-hand side, rows of 7 entries: the planner
    # takes two slices a warp (shape index 4, 1024-row chunks) and a budget of 5/4 of L2; with
    # float32 values it keeps shape 1; the powers equal the oracle's binary32 path
    A = gen.laplacian_3d(40, 36, 30)
    _, l2 = mpk.device_info()
    for vt, shape, rows, frac in ((mpk.MPK_BF16, 4, 1024, 5), (mpk.MPK_F32, 1, 512, 3)):
        dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vt)
        L = mpk.build_levels(dA, 0)
        P = mpk.plan(dA, L, p_max=8, order=mpk.ORDER_PLAN, accum=mpk.MPK_F32)
        d = P.describe()
        assert d["shape"] == shape and d["chunk_rows"] == rows and d["cache_bytes"] == l2 // 4 * frac
        pe = L.perm.cpu().numpy()
        X = gen.vector(A.n, 1, stream=409)
        Y = P.apply(torch.from_numpy(np.ascontiguousarray(X[pe])).cuda(), 8, Y=_poisoned((9, A.n, 1)))
        P.sync_status()
        assert _bits_equal(Y.cpu().numpy(), oracle.mpk_acc32(_widened(dA), X, 8)[:, pe, :])


@pytest.mark.parametrize("order", [0, 1])
def test_two_slice_shape_on_every_path(mpk, order):
    # the planner's two-slice shape (bfloat16 values, binary32 sums): powers with split levels,
    # the Chebyshev recurrence (real and complex coefficients, the second slice of a warp
    # through the recurrence's epilogue), in both orders, against the oracle's binary32 path
    A = gen.laplacian_3d(40, 36, 30)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    Aw = _widened(dA)
    L = mpk.build_levels(dA, 0)
    _, pe, ip, _ = oracle.levels(A, 0)
    X = gen.vector(A.n, 2, stream=411)
    Xin = torch.from_numpy(np.ascontiguousarray(X if order == 0 else X[pe])).cuda()
    for split in (False, True):
        P = mpk.plan(dA, L, p_max=8, nrhs=1, order=order, accum=mpk.MPK_F32, split_levels=split, shape=5,
                     cache_bytes=0 if not split else 4 << 20)
        assert P.describe()["shape"] == 4
        Y = P.apply(Xin[:, :1].contiguous(), 8, Y=_poisoned((9, A.n, 1)))
        P.sync_status()
        want = oracle.mpk_acc32(Aw, X[:, :1], 8)
        assert _bits_equal(Y.cpu().numpy(), want if order == 0 else want[:, pe, :])
    lo, hi = gen.gershgorin_bounds(A)
    scale, shift = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    P = mpk.plan(dA, L, p_max=8, nrhs=2, order=order, accum=mpk.MPK_F32, shape=5)
    assert P.describe()["shape"] == 4
    deg = 21
    cr = gen.uniform(gen.derive_seed(412), deg + 1)
    ci = gen.uniform(gen.derive_seed(413), deg + 1)
    for cim in (None, ci):
        got = P.cheb_filter(Xin, deg, cr, cim, scale=scale, shift=shift).cpu().numpy()
        P.sync_status()
        want = oracle.cheb_acc32(Aw, X, deg, cr, cim, scale=scale, shift=shift)
        assert _bits_equal(got[ip] if order == 1 else got, want)


def test_two_slice_shape_without_allocation(mpk):
    A = gen.laplacian_3d(40, 36, 30)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=8, order=mpk.ORDER_PLAN, accum=mpk.MPK_F32)
    assert P.describe()["shape"] == 4
    pe = L.perm.cpu().numpy()
    X = gen.vector(A.n, 1, stream=414)
    Xp = torch.from_numpy(np.ascontiguousarray(X[pe])).cuda()
    want = P.apply(Xp, 8)
    P.sync_status()
    Y = _poisoned((9, A.n, 1))
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    P.apply_noalloc(Xp, 8, Y, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and torch.equal(Y, want)

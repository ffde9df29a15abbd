"""CUDA path (through the C ABI) against the CPU oracle.

Bit-exact everywhere: levels, permutation and groups are integers; every floating-point
result is a row sum evaluated in stored order with one fma per entry on both sides, so
the CUDA results must equal the oracle's bit for bit (the 1e-13 relative tolerance of the
FP64 contract is therefore met with margin; it is asserted as well).
"""
import numpy as np
import pytest

import gen
import oracle
from conftest import read_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-13


@pytest.fixture(scope="module")
def mpk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_12525_gb300 as m
    m.build()
    m.load()
    return m


def _dev(A, mpk, sym=False):
    return mpk.CsrMatrix.from_host(A, is_symmetric=sym)


def _fig1():
    edges = read_golden("fig1_graph.txt")
    n = 20
    r = list(range(n)) + [u for u, v in edges] + [v for u, v in edges]
    c = list(range(n)) + [v for u, v in edges] + [u for u, v in edges]
    return gen.from_coo(n, r, c, np.arange(len(r), dtype=np.float64) * 0.25 - 3.0)


def _disconnected():
    n = 9
    e = [(0, 1), (1, 2), (3, 4), (6, 7)]
    r = list(range(n)) + [u for u, v in e] + [v for u, v in e]
    c = list(range(n)) + [v for u, v in e] + [u for u, v in e]
    return gen.from_coo(n, r, c, np.linspace(-1, 1, len(r)))


def _star_one_way(n=40):
    r = list(range(n)) + list(range(1, n))
    c = list(range(n)) + [0] * (n - 1)
    return gen.from_coo(n, r, c, np.linspace(0.5, 1.5, len(r)))


def _empty_rows():
    # rows 3 and 7 store nothing; row 5 stores only a zero
    rows = [0, 0, 1, 2, 4, 4, 5, 6, 8, 8, 9]
    cols = [0, 4, 1, 2, 4, 8, 5, 6, 8, 0, 9]
    vals = [1.5, -2.0, 1.0, 3.0, 0.5, 1.0, 0.0, -1.0, 2.0, 0.25, 1.0]
    return gen.from_coo(10, rows, cols, vals)


MATRICES = {
    "fig1": (_fig1, False),
    "lap3d_5x4x3": (lambda: gen.laplacian_3d(5, 4, 3), True),
    "lap3d_17x9x6": (lambda: gen.laplacian_3d(17, 9, 6), True),
    "lap2d_64": (lambda: gen.laplacian_2d(64, 64), True),
    "band_3000": (lambda: gen.banded_random(3000, stream=71), True),
    "int_nonsym_500": (lambda: gen.random_int_matrix(500, 5, stream=72), False),
    "disconnected": (_disconnected, False),
    "star_one_way": (_star_one_way, False),
    "empty_rows": (_empty_rows, False),
    "xxz_10": (lambda: gen.xxz_chain(10, stream=73), True),
    "single": (lambda: gen.CSR([0, 1], [0], np.array([2.0])), True),
}


def _poisoned(shape):
    return torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")


# ----------------------------------------------------------------------------- levels (a1-a3)
@pytest.mark.parametrize("name", sorted(MATRICES))
@pytest.mark.parametrize("declare_symmetric", [False, True])
def test_levels_bit_exact(mpk, name, declare_symmetric):
    make, sym = MATRICES[name]
    if declare_symmetric and not sym:
        pytest.skip("pattern not symmetric")
    A = make()
    roots = [0] if A.n < 3 else [0, A.n // 2, A.n - 1]
    for root in roots:
        L = mpk.build_levels(_dev(A, mpk, declare_symmetric), root=root)
        lo, pe, ip, lp = oracle.levels(A, root)
        assert L.num_levels == lp.size - 1
        assert np.array_equal(L.level_of.cpu().numpy(), lo)
        assert np.array_equal(L.perm.cpu().numpy(), pe)
        assert np.array_equal(L.iperm.cpu().numpy(), ip)
        assert np.array_equal(L.level_ptr.cpu().numpy(), lp)


def test_levels_fig1_against_paper(mpk):
    L = mpk.build_levels(_dev(_fig1(), mpk), 0)
    golden = dict((o, nl) for o, nl in read_golden("fig1_perm.txt"))
    assert L.iperm.cpu().numpy().tolist() == [golden[o] for o in range(20)]
    assert np.diff(L.level_ptr.cpu().numpy()).tolist() == [1, 1, 2, 3, 3, 3, 3, 2, 1, 1]


def test_levels_grid_many_levels(mpk):
    A = gen.laplacian_3d(48, 40, 33)   # 118 levels, widths vary
    L = mpk.build_levels(_dev(A, mpk, True), 0)
    i = np.arange(A.n)
    assert np.array_equal(L.level_of.cpu().numpy(), i % 48 + (i // 48) % 40 + i // (48 * 40))
    _, pe, _, lp = oracle.levels(A, 0)
    assert np.array_equal(L.perm.cpu().numpy(), pe)
    assert np.array_equal(L.level_ptr.cpu().numpy(), lp)


def test_invalid_csr_rejected(mpk):
    A = gen.laplacian_2d(5, 5)
    bad = gen.CSR(A.row_ptr, A.col.copy(), A.val)
    bad.col[3] = 25
    with pytest.raises(mpk.MpkError) as e:
        mpk.build_levels(_dev(bad, mpk), 0)
    assert e.value.status == 1
    rp = A.row_ptr.copy()
    rp[4], rp[5] = rp[5], rp[4]
    with pytest.raises(mpk.MpkError):
        mpk.build_levels(_dev(gen.CSR(rp, A.col, A.val), mpk), 0)
    with pytest.raises(mpk.MpkError):
        mpk.build_levels(_dev(A, mpk), root=25)


# ----------------------------------------------------------------------------- plan (a3-a4)
@pytest.mark.parametrize("name", ["lap3d_17x9x6", "band_3000", "int_nonsym_500", "xxz_10", "fig1"])
@pytest.mark.parametrize("cache_bytes,p_max,m", [(4000, 4, 1), (60000, 8, 2), (10**9, 3, 1), (1, 2, 4)])
def test_plan_groups_and_permuted_matrix(mpk, name, cache_bytes, p_max, m):
    make, sym = MATRICES[name]
    A = make()
    dA = _dev(A, mpk, sym)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=p_max, nrhs=m, cache_bytes=cache_bytes, chunk_rows=64)
    lo, pe, ip, lp = oracle.levels(A, 0)
    prp, pci, pva = oracle.permute(A, pe, ip)
    budget = cache_bytes // (3 * p_max + 1)
    assert P.describe()["window"] == 3 * p_max + 1
    g = oracle.groups(lp, prp, budget, val_bytes=8, m=m)
    assert np.array_equal(P.group_level_ptr.cpu().numpy(), g)
    assert np.array_equal(P.group_row_ptr.cpu().numpy(), lp[g])
    rp, ci, va = P.export_csr()
    assert np.array_equal(rp.cpu().numpy(), prp)
    assert np.array_equal(ci.cpu().numpy(), pci)
    assert np.array_equal(va.cpu().numpy().view(np.uint64), pva.view(np.uint64))
    # chunks never cross a group boundary and hold at most chunk_rows rows
    cr = P.chunk_row_ptr.cpu().numpy()
    assert cr[0] == 0 and cr[-1] == A.n and np.all(np.diff(cr) <= 64) and np.all(np.diff(cr) > 0)
    assert set(lp[g].tolist()) <= set(cr.tolist())


# ----------------------------------------------------------------------------- apply (a5-a7)
def _check_powers(Yg, Yo):
    Yg = Yg.cpu().numpy()
    assert Yg.shape == Yo.shape
    assert np.array_equal(Yg.view(np.uint64), Yo.view(np.uint64)), "not bit-identical to the oracle"
    for k in range(Yo.shape[0]):
        nrm = np.linalg.norm(Yo[k])
        if nrm > 0:
            assert np.linalg.norm(Yg[k] - Yo[k]) / nrm <= REL_TOL


@pytest.mark.parametrize("name", sorted(MATRICES))
@pytest.mark.parametrize("order", [0, 1])
def test_apply_bit_exact(mpk, name, order):
    make, sym = MATRICES[name]
    A = make()
    dA = _dev(A, mpk, sym)
    L = mpk.build_levels(dA, 0)
    p_max, m = 6, 2
    P = mpk.plan(dA, L, p_max=p_max, nrhs=m, cache_bytes=20000, order=order, chunk_rows=32)
    X = gen.vector(A.n, m, stream=81)
    _, pe, ip, _ = oracle.levels(A, 0)
    Xin = X if order == 0 else X[pe]
    Yo = oracle.mpk(A, X, p_max)
    if order == 1:
        Yo = Yo[:, pe, :]
    for p in (1, 3, p_max):
        Y = _poisoned((p + 1, A.n, m))
        P.apply(torch.from_numpy(np.ascontiguousarray(Xin)).cuda(), p, Y=Y)
        P.sync_status()
        _check_powers(Y, Yo[: p + 1])


@pytest.mark.parametrize("m", [1, 2, 4, 8])
@pytest.mark.parametrize("chunk_rows", [32, 96, 512])
def test_apply_nrhs_and_chunks(mpk, m, chunk_rows):
    A = gen.laplacian_3d(21, 13, 11)
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=8, nrhs=m, cache_bytes=300000, chunk_rows=chunk_rows)
    X = gen.vector(A.n, m, stream=82)
    Y = P.apply(torch.from_numpy(X).cuda(), 8, Y=_poisoned((9, A.n, m)))
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X, 8))


def _arrowhead(side=40, width=1500):
    # 2-D Laplacian plus a dense first row and column: row 0 stores `width` + 1 entries, so
    # its slice is wider than one shared-memory slot and its chunk is read from global memory
    A = gen.laplacian_2d(side, side)
    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    cols = np.asarray(A.col)
    vals = np.asarray(A.val)
    tgt = np.arange(1, width + 1)
    w = gen.uniform(gen.derive_seed(85), width, 0.001, 0.01)
    r = np.concatenate([rows, np.zeros(width, np.int64), tgt])
    c = np.concatenate([cols, tgt, np.zeros(width, np.int64)])
    v = np.concatenate([vals, w, w[::-1]])
    return gen.from_coo(n, r, c, v)


@pytest.mark.parametrize("m", [1, 2, 8])
@pytest.mark.parametrize("chunk_rows,cache_bytes", [(512, 1 << 30), (608, 1 << 30), (2048, 1 << 30),
                                                     (608, 2_000_000)])
def test_apply_large_chunks(mpk, m, chunk_rows, cache_bytes):
    # a 2-D Laplacian (slices at most 5 entries wide): chunks of 16 and 19 slices, cut further
    # by the shared-memory slot, so that compute warps take several slices of a unit; chunks of
    # more than 16 slices are read from global memory, the last chunk of each group is ragged,
    # and a smaller budget cuts groups short
    A = gen.laplacian_2d(160, 150)
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=8, nrhs=m, cache_bytes=cache_bytes, chunk_rows=chunk_rows, order=mpk.ORDER_PLAN)
    d = P.describe()
    cr = P.chunk_row_ptr.cpu().numpy()
    assert np.diff(cr).max() <= chunk_rows
    if cache_bytes == 1 << 30:
        assert d["num_groups"] == 1 and np.diff(cr).max() >= 16 * 32
    X = gen.vector(A.n, m, stream=84)
    pe = mpk.build_levels(dA, 0).perm.cpu().numpy()
    Xp = np.ascontiguousarray(X[pe])
    Y = P.apply(torch.from_numpy(Xp).cuda(), 8, Y=_poisoned((9, A.n, m)))
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X, 8)[:, pe, :])


@pytest.mark.parametrize("chunk_rows", [64, 1024])
def test_apply_unstaged_wide_row(mpk, chunk_rows):
    A = _arrowhead()
    assert np.diff(A.row_ptr).max() > 1000  # one slice of 32 such rows exceeds a shared-memory slot
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    X = gen.vector(A.n, 1, stream=86)
    Yo = oracle.mpk(A, X, 6)
    for order in (mpk.ORDER_ORIGINAL, mpk.ORDER_PLAN):
        P = mpk.plan(dA, L, p_max=6, cache_bytes=50000, chunk_rows=chunk_rows, order=order)
        if order == mpk.ORDER_PLAN:
            pe = L.perm.cpu().numpy()
            Y = P.apply(torch.from_numpy(np.ascontiguousarray(X[pe])).cuda(), 6, Y=_poisoned((7, A.n, 1)))
            P.sync_status()
            _check_powers(Y, Yo[:, pe, :])
        else:
            Y = P.apply(torch.from_numpy(X).cuda(), 6, Y=_poisoned((7, A.n, 1)))
            P.sync_status()
            _check_powers(Y, Yo)


def test_apply_small_config_many_groups(mpk):
    # 64x64 5-point Laplacian, p = 4 (the small configuration), groups of single levels
    A, p = gen.config_small()
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    X = gen.vector(A.n, 1, stream=1)
    for cache in (1, 5000, 0):
        P = mpk.plan(dA, L, p_max=p, cache_bytes=cache)
        Y = P.apply(torch.from_numpy(X).cuda(), p, Y=_poisoned((p + 1, A.n, 1)))
        P.sync_status()
        _check_powers(Y, oracle.mpk(A, X, p))


def test_apply_p31_and_p0(mpk):
    A = gen.row_stochastic(700, 2, stream=83)
    dA = _dev(A, mpk)
    L = mpk.build_levels(dA, 5)
    P = mpk.plan(dA, L, p_max=31, cache_bytes=4000, chunk_rows=32)
    X = np.ones((A.n, 1))
    Y = P.apply(torch.from_numpy(X).cuda(), 31)
    P.sync_status()
    assert torch.all(Y == 1.0)
    Y0 = P.apply(torch.from_numpy(X).cuda(), 0)
    assert torch.all(Y0 == 1.0) and Y0.shape == (1, A.n, 1)


def test_identity_plan_and_comparator(mpk):
    A = gen.laplacian_3d(19, 11, 7)
    dA = _dev(A, mpk, True)
    X = gen.vector(A.n, 1, stream=84)
    Yo = oracle.mpk(A, X, 7)
    P0 = mpk.plan(dA, None, p_max=7, chunk_rows=64)         # natural order, one group
    assert P0.describe()["num_groups"] == 1
    _check_powers(P0.apply(torch.from_numpy(X).cuda(), 7), Yo)
    _check_powers(P0.spmv_powers(torch.from_numpy(X).cuda(), 7), Yo)
    L = mpk.build_levels(dA, 0)
    for order in (0, 1):
        P = mpk.plan(dA, L, p_max=7, order=order, cache_bytes=50000)
        _, pe, _, _ = oracle.levels(A, 0)
        Xin = X if order == 0 else X[pe]
        want = Yo if order == 0 else Yo[:, pe, :]
        Ya = P.apply(torch.from_numpy(np.ascontiguousarray(Xin)).cuda(), 7)
        Ys = P.spmv_powers(torch.from_numpy(np.ascontiguousarray(Xin)).cuda(), 7)
        P.sync_status()
        _check_powers(Ya, want)
        _check_powers(Ys, want)
        assert torch.equal(Ya, Ys)  # level-blocked == back-to-back, bit for bit


def test_repeated_applies_reuse_plan(mpk):
    A = gen.banded_random(4000, stream=85)
    dA = _dev(A, mpk, True)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=5, cache_bytes=100000, chunk_rows=64)
    for s in range(6):
        X = gen.vector(A.n, 1, stream=200 + s)
        Y = P.apply(torch.from_numpy(X).cuda(), 1 + s % 5)
        P.sync_status()
        _check_powers(Y, oracle.mpk(A, X, 1 + s % 5))


def test_timeout_is_reported_and_plan_recovers(mpk):
    A = gen.laplacian_3d(16, 16, 16)
    dA = _dev(A, mpk, True)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=4, chunk_rows=32, cache_bytes=20000,
                 wait_limit_ns=20_000_000)
    X = torch.from_numpy(gen.vector(A.n, 1, stream=86)).cuda()
    P.debug_drop_release(chunk=3, k=1)     # nothing will ever set this flag
    P.apply(X, 4)
    with pytest.raises(mpk.MpkError) as e:
        P.sync_status()
    assert e.value.status == 4
    Y = P.apply(X, 4)                      # the next launch is unaffected
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X.cpu().numpy(), 4))


def test_bad_arguments(mpk):
    A = gen.laplacian_2d(8, 8)
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, L, p_max=0)
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, L, nrhs=3)
    with pytest.raises(mpk.MpkError) as e:
        mpk.plan(dA, L, mem_budget=1000)
    assert e.value.status == 6
    P = mpk.plan(dA, L, p_max=3)
    with pytest.raises(mpk.MpkError):
        P.apply(torch.zeros(64, dtype=torch.float64, device="cuda"), 4)
    # outputs that cannot hold what the call writes are refused by the binding
    X = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        P.apply(X, 3, Y=torch.empty((3, 64, 1), dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        P.apply(X, 2, Y=torch.empty((3, 64, 1), dtype=torch.float64))
    with pytest.raises(ValueError):
        P.cheb_filter(X, 3, np.ones(4), out=torch.empty(10, dtype=torch.float64, device="cuda"))


# ----------------------------------------------------------------------------- Chebyshev (a6')
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("degree,p_max", [(0, 4), (1, 4), (13, 4), (16, 8), (7, 31)])
def test_cheb_real_bit_exact(mpk, order, degree, p_max):
    A = gen.xxz_chain(12, stream=87)
    dA = _dev(A, mpk, True)
    lo, hi = gen.gershgorin_bounds(A)
    scale, shift = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=p_max, nrhs=2, order=order, cache_bytes=30000, chunk_rows=64)
    X = gen.vector(A.n, 2, stream=88)
    c = gen.uniform(gen.derive_seed(89), degree + 1)
    want = oracle.cheb(A, X, degree, c, scale=scale, shift=shift)
    _, pe, ip, _ = oracle.levels(A, 0)
    Xin = X if order == 0 else X[pe]
    got = P.cheb_filter(torch.from_numpy(np.ascontiguousarray(Xin)).cuda(), degree, c, scale=scale, shift=shift)
    P.sync_status()
    got = got.cpu().numpy()
    if order == 1:
        got = got[ip]
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_cheb_complex_time_step(mpk):
    A = gen.laplacian_3d(12, 10, 9)
    dA = _dev(A, mpk, True)
    lo, hi = gen.gershgorin_bounds(A)
    a, c = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    dt, M = 0.5, 24
    J = oracle.bessel_j(M, a * dt)
    coef = np.array([J[0]] + [2 * (-1j) ** k * J[k] for k in range(1, M + 1)]) * np.exp(-1j * dt * c)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, nrhs=2, cache_bytes=40000)
    psi = gen.vector(A.n, 2, stream=90)
    want = oracle.cheb(A, psi, M, coef.real.copy(), coef.imag.copy(), scale=a, shift=c)
    got = P.cheb_filter(torch.from_numpy(psi).cuda(), M, coef.real.copy(), coef.imag.copy(), scale=a, shift=c)
    P.sync_status()
    assert np.array_equal(got.cpu().numpy().view(np.uint64), want.view(np.uint64))
    # and the step is unitary to within the expansion's truncation
    z0 = psi[:, 0] + 1j * psi[:, 1]
    g = got.cpu().numpy()
    assert abs(np.linalg.norm(g[:, 0] + 1j * g[:, 1]) / np.linalg.norm(z0) - 1) < 1e-12


def test_apply_replays_from_cuda_graph(mpk):
    # launch epochs live on the device: every replay of a captured apply is a new launch
    A = gen.laplacian_3d(21, 13, 11)
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=6, cache_bytes=200000, order=mpk.ORDER_PLAN)
    pe = L.perm.cpu().numpy()
    Xs = torch.zeros((A.n, 1), dtype=torch.float64, device="cuda")
    Ys = torch.zeros((7, A.n, 1), dtype=torch.float64, device="cuda")
    P.apply(Xs, 6, Y=Ys)  # outside the capture: kernel attributes and occupancy are set up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        P.apply(Xs, 6, Y=Ys)
    for seed in (401, 402, 403):
        X = gen.vector(A.n, 1, stream=seed)
        Xs.copy_(torch.from_numpy(np.ascontiguousarray(X[pe])))
        Ys.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        P.sync_status()
        _check_powers(Ys, oracle.mpk(A, X, 6)[:, pe, :])


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("name", ["lap3d_17x9x6", "lap2d_64", "band_3000", "int_nonsym_500", "xxz_10", "empty_rows",
                                  "disconnected", "single"])
def test_apply_every_block_shape(mpk, shape, name):
    # the block shapes of the staged kernel (13 warps with 3072-entry slots, 16 warps with
    # 4608, 14 warps reading entries from global memory, input rows staged as well, and two
    # slices a warp in 9216-entry slots) give the same bits; shape 3 refuses a plan whose
    # chunks read input rows beyond a slot
    make, sym = MATRICES[name]
    A = make()
    dA = _dev(A, mpk, sym)
    L = mpk.build_levels(dA, 0)
    X = gen.vector(A.n, 2, stream=98)
    try:
        P = mpk.plan(dA, L, p_max=7, nrhs=2, cache_bytes=30000, shape=shape)
    except mpk.MpkError as e:
        assert shape == 4 and e.status == 7
        pytest.skip("input rows of a chunk exceed a shape-3 slot")
    assert P.describe()["shape"] == shape - 1
    Y = P.apply(torch.from_numpy(X).cuda(), 7, Y=_poisoned((8, A.n, 2)))
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X, 7))
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, L, p_max=3, shape=6)


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_two_slices_a_warp(mpk, m, order):
    # block shape 4 (plan option 5): 1024-row chunks of up to 32 slices, two slices for each of
    # the 16 compute warps, on matrices whose groups hold full chunks and ragged last ones
    for A in (gen.laplacian_3d(40, 40, 40), gen.banded_random(60000, stream=176), gen.laplacian_2d(300, 211)):
        dA = _dev(A, mpk, True)
        L = mpk.build_levels(dA, 0)
        pe = L.perm.cpu().numpy()
        X = gen.vector(A.n, m, stream=177)
        for cache, cr in ((0, 0), (2000000, 0), (0, 800)):
            P = mpk.plan(dA, L, p_max=8, nrhs=m, cache_bytes=cache, order=order, chunk_rows=cr, shape=5)
            d = P.describe()
            assert d["shape"] == 4 and d["chunk_rows"] == (cr or 1024)
            Xin = X if order == 0 else np.ascontiguousarray(X[pe])
            Y = P.apply(torch.from_numpy(Xin).cuda(), 8, Y=_poisoned((9, A.n, m)))
            P.sync_status()
            Yo = oracle.mpk(A, X, 8)
            _check_powers(Y, Yo if order == 0 else Yo[:, pe, :])


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("order", [0, 1])
def test_input_rows_staged_shape(mpk, m, order):
    # shape 3 on grids whose chunks' input rows fit a slot: powers, Chebyshev, several cache
    # budgets and chunk sizes (ragged last chunks, chunks over two levels), into NaN-poisoned
    # outputs; the input vector starts 8 bytes past a 16-byte boundary in one of the runs
    for A in (gen.laplacian_3d(21, 13, 11), gen.laplacian_2d(90, 70), gen.laplacian_3d(40, 40, 40)):
        dA = _dev(A, mpk, True)
        L = mpk.build_levels(dA, 0)
        pe = L.perm.cpu().numpy()
        X = gen.vector(A.n, m, stream=171)
        Yo = oracle.mpk(A, X, 8)
        built = 0
        for cache, cr in ((30000, 0), (400000, 96), (0, 288), (0, 160)):
            try:
                P = mpk.plan(dA, L, p_max=8, nrhs=m, cache_bytes=cache, order=order, chunk_rows=cr, shape=4)
            except mpk.MpkError as e:  # a chunk's input rows exceed a slot: refused, never wrong
                assert e.status == 7
                continue
            built += 1
            assert P.describe()["shape"] == 3
            Xin = X if order == 0 else np.ascontiguousarray(X[pe])
            for shift in (0, 1):
                buf = torch.zeros(A.n * m + 1, dtype=torch.float64, device="cuda")
                Xd = buf[shift:shift + A.n * m].view(A.n, m)
                Xd.copy_(torch.from_numpy(Xin))
                Y = P.apply(Xd, 8, Y=_poisoned((9, A.n, m)))
                P.sync_status()
                _check_powers(Y, Yo if order == 0 else Yo[:, pe, :])
        assert built >= 2
        if m == 2:
            lo, hi = gen.gershgorin_bounds(A)
            c = gen.uniform(gen.derive_seed(172), 20)
            P = None
            for cr in (0, 160, 96, 64):
                try:
                    P = mpk.plan(dA, L, p_max=8, nrhs=2, cache_bytes=60000, order=0, chunk_rows=cr, shape=4)
                    break
                except mpk.MpkError as e:
                    assert e.status == 7
            assert P is not None
            got = P.cheb_filter(torch.from_numpy(X).cuda(), 19, c, scale=(hi - lo) / 2 * 1.01, shift=(hi + lo) / 2)
            P.sync_status()
            want = oracle.cheb(A, X, 19, c, scale=(hi - lo) / 2 * 1.01, shift=(hi + lo) / 2)
            assert np.array_equal(got.cpu().numpy().view(np.uint64), want.view(np.uint64))


def test_automatic_block_shape(mpk):
    # rows of 7 and of 13-15 entries fill a 4608-entry slot with at least 6 of 16 slices
    # (shape 1); 27-point rows go unstaged (shape 2)
    for A, want in ((gen.laplacian_3d(30, 30, 30), 1), (gen.xxz_chain(12, stream=99), 1), (gen.stencil27(40), 2)):
        dA = _dev(A, mpk, True)
        P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=4)
        d = P.describe()
        assert d["shape"] == want and d["engine"] == 0 and d["chunk_rows"] == 32 * (16 if want == 1 else 14)


@pytest.mark.parametrize("seed", [1, 2, 0x5EED])
@pytest.mark.parametrize("name", ["lap3d_17x9x6", "band_3000", "int_nonsym_500", "disconnected", "xxz_10"])
def test_shuffled_schedules_give_the_same_bits(mpk, seed, name):
    # race-detection aid: the units of every schedule line in a seeded random order; any
    # dependency that a unit did not wait for would show up as a different bit or a NaN
    make, sym = MATRICES[name]
    A = make()
    dA = _dev(A, mpk, sym)
    L = mpk.build_levels(dA, 0)
    X = gen.vector(A.n, 2, stream=99)
    P = mpk.plan(dA, L, p_max=7, nrhs=2, cache_bytes=20000, chunk_rows=32, shuffle_seed=seed)
    Y = P.apply(torch.from_numpy(X).cuda(), 7, Y=_poisoned((8, A.n, 2)))
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X, 7))
    if A.n > 1:
        lo, hi = gen.gershgorin_bounds(A)
        c = gen.uniform(gen.derive_seed(100), 12)
        got = P.cheb_filter(torch.from_numpy(X).cuda(), 11, c, scale=(hi - lo) / 2 * 1.01 + 1e-3,
                            shift=(hi + lo) / 2).cpu().numpy()
        P.sync_status()
        want = oracle.cheb(A, X, 11, c, scale=(hi - lo) / 2 * 1.01 + 1e-3, shift=(hi + lo) / 2)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("engine", [0, 2])
def test_cheb_resume_in_pieces_and_from_a_checkpoint(mpk, order, engine):
    # the recurrence state (v_{k-1}, v_k, accumulator) at any step is a resume point: pieces
    # of the degree, and a state saved to the host and restored, give the same bits as one call
    A = gen.xxz_chain(12, stream=87)
    dA = _dev(A, mpk, True)
    lo, hi = gen.gershgorin_bounds(A)
    scale, shift = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, nrhs=2, order=order, cache_bytes=30000, engine=engine)
    X = gen.vector(A.n, 2, stream=101)
    _, pe, ip, _ = oracle.levels(A, 0)
    Xin = torch.from_numpy(np.ascontiguousarray(X if order == 0 else X[pe])).cuda()
    deg = 37
    cr = gen.uniform(gen.derive_seed(102), deg + 1)
    ci = gen.uniform(gen.derive_seed(103), deg + 1)
    whole = P.cheb_filter(Xin, deg, cr, ci, scale=scale, shift=shift).cpu().numpy()
    st = P.cheb_state()
    P.cheb_begin(Xin, st, cr[0], ci[0])
    for k0, k1 in ((0, 5), (5, 16), (16, 24)):
        P.cheb_advance(st, k0, k1, cr, ci, scale=scale, shift=shift)
    saved = st.cpu().numpy().copy()                # checkpoint at step 24
    st.fill_(float("nan"))
    st.copy_(torch.from_numpy(saved))              # restore
    P.cheb_advance(st, 24, deg, cr, ci, scale=scale, shift=shift)
    got = P.cheb_finish(st).cpu().numpy()
    P.sync_status()
    assert np.array_equal(got.view(np.uint64), whole.view(np.uint64))
    want = oracle.cheb(A, X, deg, cr, ci, scale=scale, shift=shift)
    if order == 1:
        got = got[ip]
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    with pytest.raises(mpk.MpkError):
        P.cheb_advance(st, 5, 4, cr, ci, scale=scale, shift=shift)

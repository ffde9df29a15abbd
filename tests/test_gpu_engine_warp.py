"""The warp-ticketed engine of the level-blocked kernel (plan engine MPK_ENGINE_WARP): the same
Lp-diagram order with items of 32-row slices claimed by single warps and cell-level
dependency counters.  Every row keeps its stored-order fma chain, so every result must equal
the oracle (and the staged engine) bit for bit."""
import numpy as np
import pytest

import gen
import oracle
from test_gpu_parity import MATRICES, _check_powers, _dev, _poisoned

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


@pytest.mark.parametrize("name", sorted(MATRICES))
@pytest.mark.parametrize("order", [0, 1])
def test_warp_apply_bit_exact(mpk, name, order):
    make, sym = MATRICES[name]
    A = make()
    dA = _dev(A, mpk, sym)
    L = mpk.build_levels(dA, 0)
    p_max, m = 6, 2
    P = mpk.plan(dA, L, p_max=p_max, nrhs=m, cache_bytes=20000, order=order, engine=mpk.ENGINE_WARP)
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
@pytest.mark.parametrize("cache_bytes", [30000, 300000, 1 << 30])
def test_warp_nrhs_and_budgets(mpk, m, cache_bytes):
    A = gen.laplacian_3d(21, 13, 11)
    dA = _dev(A, mpk, True)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, nrhs=m, cache_bytes=cache_bytes, engine=mpk.ENGINE_WARP)
    X = gen.vector(A.n, m, stream=82)
    Y = P.apply(torch.from_numpy(X).cuda(), 8, Y=_poisoned((9, A.n, m)))
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X, 8))


def test_warp_identity_plan_and_p31(mpk):
    A = gen.banded_random(4000, stream=91, per_row=6)
    dA = _dev(A, mpk, True)
    X = gen.vector(A.n, 1, stream=92)
    P0 = mpk.plan(dA, None, p_max=5, engine=mpk.ENGINE_WARP)  # one group: p dependent sweeps
    _check_powers(P0.apply(torch.from_numpy(X).cuda(), 5, Y=_poisoned((6, A.n, 1))), oracle.mpk(A, X, 5))
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=31, cache_bytes=50000, engine=mpk.ENGINE_WARP)
    _check_powers(P.apply(torch.from_numpy(X).cuda(), 31, Y=_poisoned((32, A.n, 1))), oracle.mpk(A, X, 31))
    P.sync_status()


@pytest.mark.parametrize("vt", ["f32", "bf16"])
@pytest.mark.parametrize("m", [1, 2])
def test_warp_narrow_values_match_staged(mpk, vt, m):
    A = gen.banded_random(20000, stream=93, per_row=7, band_frac=0.01)
    code = {"f32": mpk.MPK_F32, "bf16": mpk.MPK_BF16}[vt]
    dA = mpk.CsrMatrix.from_host(A, value_type=code)
    L = mpk.build_levels(dA, 0)
    X = torch.from_numpy(gen.vector(A.n, m, stream=94)).cuda()
    Ys = mpk.plan(dA, L, p_max=6, nrhs=m, cache_bytes=200000).apply(X, 6)
    Pw = mpk.plan(dA, L, p_max=6, nrhs=m, cache_bytes=200000, engine=mpk.ENGINE_WARP)
    Yw = Pw.apply(X, 6, Y=_poisoned((7, A.n, m)))
    Pw.sync_status()
    assert torch.equal(Ys, Yw)
    widened = gen.CSR(dA.row_ptr.cpu().numpy(), dA.col.cpu().numpy(), dA.val.double().cpu().numpy())
    _check_powers(Yw, oracle.mpk(widened, X.cpu().numpy(), 6))


@pytest.mark.parametrize("order", [0, 1])
def test_warp_cheb_real_and_complex(mpk, order):
    A = gen.xxz_chain(12, stream=87)
    dA = _dev(A, mpk, True)
    lo, hi = gen.gershgorin_bounds(A)
    scale, shift = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, nrhs=2, order=order, cache_bytes=30000,
                 engine=mpk.ENGINE_WARP)
    X = gen.vector(A.n, 2, stream=88)
    _, pe, ip, _ = oracle.levels(A, 0)
    Xin = torch.from_numpy(np.ascontiguousarray(X if order == 0 else X[pe])).cuda()
    for degree in (0, 1, 13, 16):
        c = gen.uniform(gen.derive_seed(89), degree + 1)
        want = oracle.cheb(A, X, degree, c, scale=scale, shift=shift)
        got = P.cheb_filter(Xin, degree, c, scale=scale, shift=shift).cpu().numpy()
        P.sync_status()
        if order == 1:
            got = got[ip]
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), degree
    ci = gen.uniform(gen.derive_seed(95), 17)
    cr = gen.uniform(gen.derive_seed(96), 17)
    want = oracle.cheb(A, X, 16, cr, ci, scale=scale, shift=shift)
    got = P.cheb_filter(Xin, 16, cr, ci, scale=scale, shift=shift).cpu().numpy()
    if order == 1:
        got = got[ip]
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_warp_level_capped_dlb(mpk):
    from paper_2405_12525_gb300.dlb import DlbMpk
    A = gen.laplacian_3d(20, 18, 16)
    X = gen.vector(A.n, 2, stream=97)
    D = DlbMpk(A, 3, 8, nrhs=2, engine=mpk.ENGINE_WARP)
    got = D.apply(torch.from_numpy(X).cuda()).cpu().numpy()
    assert np.array_equal(got, oracle.mpk(A, X, 8))


def test_warp_graph_replay_and_repeats(mpk):
    A = gen.laplacian_3d(21, 13, 11)
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=6, cache_bytes=200000, order=mpk.ORDER_PLAN, engine=mpk.ENGINE_WARP)
    pe = L.perm.cpu().numpy()
    Xs = torch.zeros((A.n, 1), dtype=torch.float64, device="cuda")
    Ys = torch.zeros((7, A.n, 1), dtype=torch.float64, device="cuda")
    P.apply(Xs, 6, Y=Ys)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        P.apply(Xs, 6, Y=Ys)
    for seed in (411, 412, 413):
        X = gen.vector(A.n, 1, stream=seed)
        Xs.copy_(torch.from_numpy(np.ascontiguousarray(X[pe])))
        Ys.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        _check_powers(Ys, oracle.mpk(A, X, 6)[:, pe, :])
    for p in (6, 2, 5):  # shorter and longer launches in turn reuse the counters
        X = gen.vector(A.n, 1, stream=420 + p)
        Y = P.apply(torch.from_numpy(np.ascontiguousarray(X[pe])).cuda(), p, Y=_poisoned((p + 1, A.n, 1)))
        _check_powers(Y, oracle.mpk(A, X, p)[:, pe, :])
    P.sync_status()


def test_warp_engine_rejected_for_batch_and_bad_value(mpk):
    A = gen.laplacian_2d(20, 20)
    dA = _dev(A, mpk, True)
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, mpk.build_levels(dA, 0), p_max=3, engine=7)
    # a batch plan is built with the staged engine only
    import ctypes as C
    lib = mpk.load()
    o = mpk._Opts()
    lib.mpk_plan_opts_default(C.byref(o))
    assert o.engine == mpk.ENGINE_STAGED


def test_warp_timeout_is_reported_and_plan_recovers(mpk):
    # one chunk never counts its slices at power 1: every warp waiting on it gives up after the
    # plan's wait limit, the launch ends with MPK_ERR_TIMEOUT, and the next launch is unaffected
    A = gen.laplacian_3d(16, 16, 16)
    dA = _dev(A, mpk, True)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=4, cache_bytes=20000, wait_limit_ns=20_000_000,
                 engine=mpk.ENGINE_WARP)
    X = torch.from_numpy(gen.vector(A.n, 1, stream=86)).cuda()
    P.debug_drop_release(chunk=3, k=1)
    P.apply(X, 4)
    with pytest.raises(mpk.MpkError) as e:
        P.sync_status()
    assert e.value.status == 4
    Y = P.apply(X, 4)
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X.cpu().numpy(), 4))


# ----------------------------------------------------------------------------- sweep engine
@pytest.mark.parametrize("name", sorted(MATRICES))
@pytest.mark.parametrize("order", [0, 1])
def test_sweep_apply_bit_exact(mpk, name, order):
    make, sym = MATRICES[name]
    A = make()
    dA = _dev(A, mpk, sym)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=6, nrhs=2, cache_bytes=20000, order=order, engine=mpk.ENGINE_SWEEP)
    assert P.describe()["engine"] == mpk.ENGINE_SWEEP
    X = gen.vector(A.n, 2, stream=81)
    _, pe, ip, _ = oracle.levels(A, 0)
    Yo = oracle.mpk(A, X, 6)
    if order == 1:
        Yo = Yo[:, pe, :]
    Xin = torch.from_numpy(np.ascontiguousarray(X if order == 0 else X[pe])).cuda()
    for p in (1, 4, 6):
        Y = P.apply(Xin, p, Y=_poisoned((p + 1, A.n, 2)))
        P.sync_status()
        _check_powers(Y, Yo[: p + 1])
    if order == 1:
        Y = _poisoned((7, A.n, 2))
        P.apply_noalloc(Xin, 6, Y)
        _check_powers(Y, Yo)


@pytest.mark.parametrize("order", [0, 1])
def test_sweep_cheb_bit_exact(mpk, order):
    A = gen.xxz_chain(12, stream=87)
    dA = _dev(A, mpk, True)
    lo, hi = gen.gershgorin_bounds(A)
    scale, shift = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, nrhs=2, order=order, engine=mpk.ENGINE_SWEEP)
    X = gen.vector(A.n, 2, stream=88)
    _, pe, ip, _ = oracle.levels(A, 0)
    Xin = torch.from_numpy(np.ascontiguousarray(X if order == 0 else X[pe])).cuda()
    cr = gen.uniform(gen.derive_seed(96), 21)
    ci = gen.uniform(gen.derive_seed(95), 21)
    for im in (None, ci):
        want = oracle.cheb(A, X, 20, cr, im, scale=scale, shift=shift)
        got = P.cheb_filter(Xin, 20, cr, im, scale=scale, shift=shift).cpu().numpy()
        P.sync_status()
        if order == 1:
            got = got[ip]
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_sweep_engine_rejected_for_level_capped(mpk):
    A = gen.laplacian_2d(20, 20)
    dA = _dev(A, mpk, True)
    L = mpk.build_levels_from(dA, [0, 7])
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, L, p_max=3, order=mpk.ORDER_PLAN, level_capped=True, engine=mpk.ENGINE_SWEEP)


def test_autotuner_plan_candidates(mpk):
    from paper_2405_12525_gb300 import autotune
    A = gen.laplacian_3d(24, 20, 18)
    dA = _dev(A, mpk, True)
    L = mpk.build_levels(dA, 0)
    pe = L.perm.cpu().numpy()
    X = gen.vector(A.n, 1, stream=97)
    Xp = torch.from_numpy(np.ascontiguousarray(X[pe])).cuda()
    P, report = autotune.tune_plan(dA, L, 5, Xp, candidates={"cache_bytes": [100000, 1 << 22], "chunk_rows": [0]})
    assert len(report) == 3 and any(opts.get("engine") == "sweep" for _, opts in report)
    assert all(report[i][0] <= report[i + 1][0] for i in range(len(report) - 1))
    Y = P.apply(Xp, 5, Y=_poisoned((6, A.n, 1)))
    P.sync_status()
    _check_powers(Y, oracle.mpk(A, X, 5)[:, pe, :])

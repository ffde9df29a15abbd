"""DLB-MPK (Sec. 5, Alg. 2) with all partitions on one device, against the oracle.

The local problems keep every row's entries in stored order, so each power of each row is the
same fma sequence as in the single-matrix MPK: the assembled result must equal oracle.mpk bit
for bit, for DLB-MPK and for TRAD alike.  The pieces are pinned on their own as well: levels
from the halo rows against host BFS distances, the level-capped plan's per-row power caps,
the row-range SpMV and the gather.
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


def _two_components():
    # two disjoint 2-D grids: a partition may hold rows no halo row reaches
    a = gen.laplacian_2d(9, 7)
    n = 2 * a.n
    rows = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    r = np.concatenate([rows, rows + a.n])
    c = np.concatenate([a.col, a.col + a.n])
    v = np.concatenate([a.val, a.val * 0.5])
    return gen.from_coo(n, r, c, v)


CASES = {
    "lap3d": lambda: gen.laplacian_3d(20, 18, 16),
    "banded": lambda: gen.banded_random(30000, stream=41, per_row=7, band_frac=0.002),
    "stencil27": lambda: gen.stencil27(14),
    "xxz": lambda: gen.xxz_chain(12, stream=42),
    "two_components": _two_components,
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("parts", [1, 2, 3, 5])
def test_dlb_equals_oracle_bitwise(mpk, name, parts):
    from paper_2405_12525_gb300.dlb import DlbMpk
    A = CASES[name]()
    for p_m, m in ((4, 1), (8, 2)):
        X = gen.vector(A.n, m, stream=43)
        want = oracle.mpk(A, X, p_m)
        D = DlbMpk(A, parts, p_m, nrhs=m)
        Xd = torch.from_numpy(X).cuda()
        got = D.apply(Xd).cpu().numpy()
        assert np.array_equal(got, want), (name, parts, p_m, np.argwhere(got != want)[:5])
        got_t = D.trad(Xd).cpu().numpy()
        assert np.array_equal(got_t, want)
        assert 0.0 <= D.overhead <= 1.0


def test_dlb_p1_and_small_cache(mpk):
    from paper_2405_12525_gb300.dlb import DlbMpk
    A = gen.laplacian_3d(24, 24, 24)
    X = gen.vector(A.n, 1, stream=44)
    for p_m, cache in ((1, 0), (6, 1 << 20)):
        D = DlbMpk(A, 4, p_m, cache_bytes=cache)
        assert np.array_equal(D.apply(torch.from_numpy(X).cuda()).cpu().numpy(), oracle.mpk(A, X, p_m))


def test_levels_from_halo_are_boundary_distances(mpk):
    from paper_2405_12525_gb300 import dlb
    for A, parts in ((gen.laplacian_3d(16, 16, 16), 3), (gen.banded_random(20000, 45, 6, 0.003), 4),
                     (_two_components(), 2)):
        b = dlb.partition_rows(A.n, parts, A.row_ptr)
        for i in range(parts):
            pb = dlb.local_problem(A.row_ptr, A.col, A.val, int(b[i]), int(b[i + 1]), b)
            if pb["nh"] == 0:
                continue
            n_loc = pb["nl"] + pb["nh"]
            dA = mpk.CsrMatrix(torch.from_numpy(pb["row_ptr"]).cuda(), torch.from_numpy(pb["col"]).cuda(),
                               torch.from_numpy(np.asarray(pb["val"], dtype=np.float64)).cuda())
            L = mpk.build_levels_from(dA, np.arange(pb["nl"], n_loc))
            lev = L.level_of.cpu().numpy()
            d = dlb.boundary_distance(pb)
            reach = d >= 0
            assert np.array_equal(lev[:pb["nl"]][reach], d[reach])
            assert np.all(lev[pb["nl"]:] == 0)
            assert np.all(lev[:pb["nl"]][~reach] >= 1)
            lp = L.level_ptr.cpu().numpy()
            assert lp[1] == pb["nh"] and np.all(np.diff(lp) > 0)


def test_build_levels_from_rejects_bad_roots(mpk):
    A = gen.laplacian_2d(6, 6)
    dA = mpk.CsrMatrix.from_host(A)
    for roots in ([3, 2], [1, 1], [-1], [36], []):
        with pytest.raises(mpk.MpkError):
            mpk.build_levels_from(dA, roots)


@pytest.mark.parametrize("p", [2, 5])
def test_level_capped_plan_caps_each_row(mpk, p):
    # rows of level L hold powers 0..min(L, p) equal to the oracle's, higher powers untouched
    A = gen.laplacian_2d(40, 31)
    roots = np.array([0, 17, 600, 1200], dtype=np.int32)
    dA = mpk.CsrMatrix.from_host(A)
    L = mpk.build_levels_from(dA, roots)
    P = mpk.plan(dA, L, p_max=p, order=mpk.ORDER_PLAN, level_capped=True)
    perm = L.perm.cpu().numpy()
    lev = L.level_of.cpu().numpy()[perm]
    X = gen.vector(A.n, 1, stream=46)
    want = oracle.mpk(A, X, p)[:, perm]
    for noalloc in (False, True):
        Y = torch.full((p + 1, A.n, 1), float("nan"), dtype=torch.float64, device="cuda")
        Xp = torch.from_numpy(X[perm]).cuda()
        P.apply_noalloc(Xp, p, Y) if noalloc else P.apply(Xp, p, Y=Y)
        got = Y.cpu().numpy()
        for k in range(p + 1):
            have = np.minimum(lev, p) >= k
            assert np.array_equal(got[k][have], want[k][have]), (noalloc, k)
            assert np.all(np.isnan(got[k][~have]))


def test_level_capped_needs_levels(mpk):
    A = gen.laplacian_2d(6, 6)
    dA = mpk.CsrMatrix.from_host(A)
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, None, p_max=3, level_capped=True)
    L = mpk.build_levels_from(dA, [0, 5])
    with pytest.raises(mpk.MpkError):
        mpk.plan(dA, L, p_max=3, level_capped=True)  # original order would scatter partial powers
    P = mpk.plan(dA, L, p_max=3, order=mpk.ORDER_PLAN, level_capped=True)
    X = torch.zeros((A.n, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(mpk.MpkError):
        P.cheb_filter(X, 4, np.ones(5))


def test_spmv_rows_and_gather(mpk):
    A = gen.banded_random(5000, stream=47, per_row=9)
    dA = mpk.CsrMatrix.from_host(A)
    L = mpk.build_levels(dA, 0)
    P = mpk.plan(dA, L, p_max=2, nrhs=4, order=mpk.ORDER_PLAN)
    perm = L.perm.cpu().numpy()
    X = gen.vector(A.n, 4, stream=48)[perm]
    want = oracle.mpk(A, gen.vector(A.n, 4, stream=48), 1)[1][perm]
    for lo, hi in ((0, A.n), (0, 0), (1, 2), (37, 4001), (4990, 5000)):
        Y = torch.full((A.n, 4), -7.0, dtype=torch.float64, device="cuda")
        P.spmv_rows(lo, hi, torch.from_numpy(X).cuda(), Y)
        got = Y.cpu().numpy()
        assert np.array_equal(got[lo:hi], want[lo:hi])
        assert np.all(got[:lo] == -7.0) and np.all(got[hi:] == -7.0)
    with pytest.raises(mpk.MpkError):
        P.spmv_rows(10, 5, torch.from_numpy(X).cuda(), Y)
    with pytest.raises(mpk.MpkError):
        P.spmv_rows(0, A.n + 1, torch.from_numpy(X).cuda(), Y)
    src = torch.from_numpy(gen.vector(1000, 4, stream=49)).cuda()
    idx = np.array(gen.splitmix64(50, 3000) % np.uint64(1000), dtype=np.int32)
    out = torch.empty((3000, 4), dtype=torch.float64, device="cuda")
    mpk.gather_rows(src, torch.from_numpy(idx).cuda(), out)
    assert np.array_equal(out.cpu().numpy(), src.cpu().numpy()[idx])


def test_spmv_rows_multi_and_copy_rows(mpk):
    mats = [gen.banded_random(3000, stream=51, per_row=5), gen.laplacian_3d(12, 11, 10), gen.stencil27(9)]
    plans, Xs, Ys, wants, ranges = [], [], [], [], [(5, 2900), (0, 1320), (100, 101)]
    for i, A in enumerate(mats):
        dA = mpk.CsrMatrix.from_host(A)
        L = mpk.build_levels(dA, 0)
        plans.append(mpk.plan(dA, L, p_max=2, nrhs=2, order=mpk.ORDER_PLAN))
        perm = L.perm.cpu().numpy()
        X = gen.vector(A.n, 2, stream=52 + i)
        Xs.append(torch.from_numpy(X[perm]).cuda())
        Ys.append(torch.full((A.n, 2), 3.5, dtype=torch.float64, device="cuda"))
        wants.append(oracle.mpk(A, X, 1)[1][perm])
    mpk.spmv_rows_multi(plans, [r[0] for r in ranges], [r[1] for r in ranges], Xs, Ys)
    for (lo, hi), Y, want in zip(ranges, Ys, wants):
        got = Y.cpu().numpy()
        assert np.array_equal(got[lo:hi], want[lo:hi])
        assert np.all(got[:lo] == 3.5) and np.all(got[hi:] == 3.5)
    mpk.spmv_rows_multi([], [], [], [], [])  # nothing to do
    A = mats[0]
    dA = mpk.CsrMatrix.from_host(A)
    P1 = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=2, nrhs=1, order=mpk.ORDER_PLAN)
    x1 = torch.zeros((A.n, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(mpk.MpkError):  # segments with different nrhs
        mpk.spmv_rows_multi([plans[0], P1], [0, 0], [10, 10], [Xs[0], x1], [Ys[0], x1])
    with pytest.raises(mpk.MpkError):
        mpk.spmv_rows_multi([P1] * 33, [0] * 33, [1] * 33, [x1] * 33, [x1] * 33)
    with pytest.raises(mpk.MpkError):
        mpk.spmv_rows_multi([P1], [0], [A.n + 1], [x1], [x1])
    # indexed copy within one buffer: distinct destinations outside the sources
    buf = torch.from_numpy(gen.vector(4000, 2, stream=55)).cuda()
    ref = buf.cpu().numpy().copy()
    src = np.array(gen.splitmix64(56, 1500) % np.uint64(2000), dtype=np.int64)
    dst = 2000 + np.array(gen.splitmix64(57, 2000) % np.uint64(2000), dtype=np.int64)
    dst = np.unique(dst)[:1500]
    src = src[:dst.size]
    mpk.copy_rows(buf, torch.from_numpy(src).cuda(), buf, torch.from_numpy(dst).cuda())
    ref[dst] = ref[src]
    assert np.array_equal(buf.cpu().numpy(), ref)


def test_dlb_resident_run_matches_apply(mpk):
    from paper_2405_12525_gb300.dlb import DlbMpk
    A = gen.laplacian_3d(18, 18, 18)
    X = gen.vector(A.n, 1, stream=58)
    want = oracle.mpk(A, X, 6)
    D = DlbMpk(A, 3, 6)
    Xd = torch.from_numpy(X).cuda()
    D.load(Xd)
    for trad in (False, True):
        D.run_trad() if trad else D.run()
        Y = torch.empty((7, A.n, 1), dtype=torch.float64, device="cuda")
        D.store(Y)
        assert np.array_equal(Y.cpu().numpy(), want)
    # replayed from a CUDA graph
    g = torch.cuda.CUDAGraph()
    Y = torch.empty((7, A.n, 1), dtype=torch.float64, device="cuda")
    D.apply(Xd, Y)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        D.apply(Xd, Y)
    Y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(Y.cpu().numpy(), want)

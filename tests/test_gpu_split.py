"""Bulky levels split (plan option split_levels): groups against the oracle's rule, and every
result bit for bit against the oracle with the units in exact-dependency wave order."""
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


def _poisoned(shape):
    return torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")


def _bits_equal(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


def _star(k=40):
    r = list(range(k + 1)) + [0] * k + list(range(1, k + 1))
    c = list(range(k + 1)) + list(range(1, k + 1)) + [0] * k
    return gen.from_coo(k + 1, r, c, np.linspace(1.0, 2.0, len(r)))


MATS = {
    "lap3d_14x11x9": (lambda: gen.laplacian_3d(14, 11, 9), True),
    "lap2d_64": (lambda: gen.laplacian_2d(64, 64), True),
    "band_3000": (lambda: gen.banded_random(3000, stream=71), True),
    "xxz_10": (lambda: gen.xxz_chain(10, stream=73), True),
    "star_40": (_star, True),
    "int_nonsym_500": (lambda: gen.random_int_matrix(500, 5, stream=72), False),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("cache_bytes", [20000, 200000])
@pytest.mark.parametrize("m", [1, 2])
def test_split_groups_and_powers(mpk, name, cache_bytes, m):
    make, sym = MATS[name]
    A = make()
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=sym)
    L = mpk.build_levels(dA, 0)
    p_max = 6
    lo, pe, ip, lp = oracle.levels(A, 0)
    prp, pci, pva = oracle.permute(A, pe, ip)
    budget = cache_bytes // (3 * p_max + 1)
    want_groups = oracle.groups_split(lp, prp, budget, val_bytes=8, m=m)
    X = gen.vector(A.n, m, stream=501)
    Yo = oracle.mpk(A, X, p_max)
    for order in (0, 1):
        P = mpk.plan(dA, L, p_max=p_max, nrhs=m, cache_bytes=cache_bytes, order=order, split_levels=True)
        d = P.describe()
        assert d["split_levels"] == 1
        assert np.array_equal(P.group_row_ptr.cpu().numpy(), want_groups)
        Xin = X if order == 0 else np.ascontiguousarray(X[pe])
        for p in (1, 3, p_max):
            Y = P.apply(torch.from_numpy(Xin).cuda(), p, Y=_poisoned((p + 1, A.n, m)))
            P.sync_status()
            want = Yo[: p + 1] if order == 0 else Yo[: p + 1][:, pe, :]
            assert _bits_equal(Y.cpu().numpy(), want), (order, p)
    # the split groups really break the +-1 rule somewhere: the waves are needed
    assert want_groups.size - 1 >= oracle.groups(lp, prp, budget, m=m).size - 1


@pytest.mark.parametrize("seed", [3, 0xBEEF])
@pytest.mark.parametrize("name", ["lap3d_14x11x9", "band_3000", "star_40"])
def test_split_shuffled_waves_and_chebyshev(mpk, seed, name):
    make, sym = MATS[name]
    A = make()
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=sym)
    L = mpk.build_levels(dA, 0)
    X = gen.vector(A.n, 2, stream=502)
    P = mpk.plan(dA, L, p_max=7, nrhs=2, cache_bytes=15000, chunk_rows=32, split_levels=True, shuffle_seed=seed)
    Y = P.apply(torch.from_numpy(X).cuda(), 7, Y=_poisoned((8, A.n, 2)))
    P.sync_status()
    assert _bits_equal(Y.cpu().numpy(), oracle.mpk(A, X, 7))
    lo, hi = gen.gershgorin_bounds(A)
    c = gen.uniform(gen.derive_seed(503), 18)
    sc, sh = (hi - lo) / 2 * 1.01 + 1e-3, (hi + lo) / 2
    got = P.cheb_filter(torch.from_numpy(X).cuda(), 17, c, scale=sc, shift=sh).cpu().numpy()
    P.sync_status()
    assert _bits_equal(got, oracle.cheb(A, X, 17, c, scale=sc, shift=sh))


def test_split_with_sweep_engine_and_binary32_accumulation(mpk):
    A = gen.laplacian_3d(16, 12, 10)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    L = mpk.build_levels(dA, 0)
    Aw = gen.CSR(dA.row_ptr.cpu().numpy(), dA.col.cpu().numpy(), dA.val.double().cpu().numpy())
    X = gen.vector(A.n, 1, stream=504)
    want = oracle.mpk_acc32(Aw, X, 6)
    for engine in (0, 2):
        P = mpk.plan(dA, L, p_max=6, cache_bytes=30000, engine=engine, split_levels=True, accum=mpk.MPK_F32)
        Y = P.apply(torch.from_numpy(X).cuda(), 6, Y=_poisoned((7, A.n, 1)))
        P.sync_status()
        assert _bits_equal(Y.cpu().numpy(), want)


def test_split_rejected_combinations(mpk):
    A = gen.laplacian_2d(20, 20)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True)
    L = mpk.build_levels(dA, 0)
    for kw in ({"engine": 1}, {"level_capped": True, "order": 1}):
        with pytest.raises(mpk.MpkError) as e:
            mpk.plan(dA, L, p_max=3, split_levels=True, **kw)
        assert e.value.status == 1
    with pytest.raises(mpk.MpkError) as e:
        mpk.plan(dA, None, p_max=3, split_levels=True)
    assert e.value.status == 1

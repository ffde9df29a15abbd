"""Value types (a6 precision): matrices stored as float32 or bfloat16, widened exactly to
float64 inside the kernels, accumulated in float64.

The oracle runs on the widened values (torch's own float32/bfloat16 -> float64 conversion of
the stored tensor, independent of the library), so every result must match it bit for bit;
the error of the narrow storage against the float64 matrix is stated per power.
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
    """The CSR with the stored (narrow) values widened to float64 by torch."""
    return gen.CSR(dA.row_ptr.cpu().numpy(), dA.col.cpu().numpy(), dA.val.double().cpu().numpy())


def _poisoned(shape):
    return torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")


def _bits_equal(a, b):
    return np.array_equal(np.asarray(a).view(np.uint64), np.asarray(b).view(np.uint64))


def test_widen_values_special_classes(mpk):
    f32 = np.array([0.0, -0.0, 1.0, -2.5, 1e-45, -1e-45, 1.1754942e-38, 1.1754944e-38, 3.4028235e38, -3.4028235e38,
                    np.inf, -np.inf, 6.0, -1.0, 0.1, 123456.789, 2.0 ** -130, -(2.0 ** -140)], dtype=np.float32)
    nan_bits = np.array([0x7fc00000, 0xffc00001, 0x7fa12345], dtype=np.uint32).view(np.float32)
    rnd = gen.normal(gen.derive_seed(301), 4096).astype(np.float32) * np.float32(1e3)
    vals = np.concatenate([f32, nan_bits, rnd])
    got = mpk.widen_values(torch.from_numpy(vals).cuda()).cpu().numpy()
    with np.errstate(invalid="ignore"):  # the signaling NaN is quieted, as IEEE 754 requires
        want = vals.astype(np.float64)
    assert _bits_equal(got, want)  # numpy's IEEE widening, NaN payloads included
    # bfloat16: the stored bits are the upper half of a float32
    bf_bits = (vals.view(np.uint32) >> 16).astype(np.uint16)
    t = torch.from_numpy(bf_bits.view(np.int16)).cuda().view(torch.bfloat16)
    got = mpk.widen_values(t).cpu().numpy()
    with np.errstate(invalid="ignore"):
        want = (bf_bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert _bits_equal(got, want)


MATS = {
    "lap3d_21x13x11": lambda: gen.laplacian_3d(21, 13, 11),
    "band_3000": lambda: gen.banded_random(3000, stream=71),
    "xxz_10": lambda: gen.xxz_chain(10, stream=73),
    "stencil27_9": lambda: gen.stencil27(9),
}


@pytest.mark.parametrize("name", sorted(MATS))
@pytest.mark.parametrize("vtype", ["f32", "bf16"])
@pytest.mark.parametrize("order", [0, 1])
def test_apply_value_types_bit_exact(mpk, name, vtype, order):
    A = MATS[name]()
    vt = {"f32": mpk.MPK_F32, "bf16": mpk.MPK_BF16}[vtype]
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vt)
    Aw = _widened(dA)
    L = mpk.build_levels(dA, 0)
    p, m = 6, 2
    P = mpk.plan(dA, L, p_max=p, nrhs=m, cache_bytes=60000, chunk_rows=96, order=order)
    X = gen.vector(A.n, m, stream=302)
    Yo = oracle.mpk(Aw, X, p)
    if order == mpk.ORDER_PLAN:
        pe = L.perm.cpu().numpy()
        Y = P.apply(torch.from_numpy(np.ascontiguousarray(X[pe])).cuda(), p, Y=_poisoned((p + 1, A.n, m)))
        Yo = Yo[:, pe, :]
    else:
        Y = P.apply(torch.from_numpy(X).cuda(), p, Y=_poisoned((p + 1, A.n, m)))
    P.sync_status()
    assert _bits_equal(Y.cpu().numpy(), Yo)
    # the plain comparator uses the same stored values
    Y2 = P.spmv_powers(torch.from_numpy(X if order == 0 else np.ascontiguousarray(X[L.perm.cpu().numpy()])).cuda(), p)
    P.sync_status()
    assert _bits_equal(Y2.cpu().numpy(), Yo)


@pytest.mark.parametrize("name", ["lap3d_21x13x11", "stencil27_9"])
def test_bf16_exact_stencil_equals_fp64(mpk, name):
    # {6, -1} and {26, -1} are bfloat16 numbers: the 2-byte matrix gives the float64 results
    A = MATS[name]()
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_BF16)
    assert _bits_equal(dA.val.double().cpu().numpy(), A.val)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, cache_bytes=100000)
    X = gen.vector(A.n, 1, stream=303)
    Y = P.apply(torch.from_numpy(X).cuda(), 8, Y=_poisoned((9, A.n, 1)))
    P.sync_status()
    assert _bits_equal(Y.cpu().numpy(), oracle.mpk(A, X, 8))


@pytest.mark.parametrize("vtype,val_bytes", [("f32", 4), ("bf16", 2)])
def test_group_rule_uses_value_bytes(mpk, vtype, val_bytes):
    A = gen.laplacian_3d(17, 9, 6)
    vt = {"f32": mpk.MPK_F32, "bf16": mpk.MPK_BF16}[vtype]
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vt)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=4, cache_bytes=30000)
    lo, pe, ip, lp = oracle.levels(A, 0)
    prp, _, _ = oracle.permute(A, pe, ip)
    g = oracle.groups(lp, prp, 30000 // (3 * 4 + 1), val_bytes=val_bytes, m=1)
    assert np.array_equal(P.group_level_ptr.cpu().numpy(), g)
    rp, ci, va = P.export_csr()
    _, _, pva = oracle.permute(_widened(dA), pe, ip)
    assert _bits_equal(va.cpu().numpy(), pva)


def test_cheb_f32_values_bit_exact(mpk):
    A = gen.xxz_chain(10, stream=73)
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=mpk.MPK_F32)
    Aw = _widened(dA)
    lo, hi = gen.gershgorin_bounds(Aw)
    a, c = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    M = 20
    J = oracle.bessel_j(M, a * 0.4)
    coef = np.array([J[0]] + [2 * (-1j) ** k * J[k] for k in range(1, M + 1)]) * np.exp(-0.4j * c)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, nrhs=2, cache_bytes=40000)
    psi = gen.vector(A.n, 2, stream=304)
    want = oracle.cheb(Aw, psi, M, coef.real.copy(), coef.imag.copy(), scale=a, shift=c)
    got = P.cheb_filter(torch.from_numpy(psi).cuda(), M, coef.real.copy(), coef.imag.copy(), scale=a, shift=c)
    P.sync_status()
    assert _bits_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("vtype,bound", [("f32", 1e-6), ("bf16", 2e-2)])
def test_narrow_storage_error_stated(mpk, vtype, bound, capsys):
    # N(0,1) values are not representable: the error against the float64 matrix is that of
    # the rounded values, stated per power (relative 2-norm)
    A = gen.banded_random(3000, stream=71)
    vt = {"f32": mpk.MPK_F32, "bf16": mpk.MPK_BF16}[vtype]
    dA = mpk.CsrMatrix.from_host(A, is_symmetric=True, value_type=vt)
    P = mpk.plan(dA, mpk.build_levels(dA, 0), p_max=8, cache_bytes=60000)
    X = gen.vector(A.n, 1, stream=305)
    Y = P.apply(torch.from_numpy(X).cuda(), 8).cpu().numpy()
    P.sync_status()
    Yo = oracle.mpk(A, X, 8)
    err = [float(np.linalg.norm(Y[k] - Yo[k]) / np.linalg.norm(Yo[k])) for k in range(1, 9)]
    with capsys.disabled():
        print(f"\n{vtype} storage, banded N(0,1) n=3000: relative error per power 1..8 = "
              + ", ".join(f"{e:.2e}" for e in err))
    assert max(err) < bound


@pytest.mark.parametrize("bad", [1e-40, float("inf"), float("nan")])
def test_narrow_storage_rejects_special_values(mpk, bad):
    A = gen.laplacian_2d(8, 8)
    v = A.val.copy()
    v[5] = bad
    A2 = gen.CSR(A.row_ptr, A.col, v)
    dA = mpk.CsrMatrix.from_host(A2, is_symmetric=True, value_type=mpk.MPK_F32)
    with pytest.raises(mpk.MpkError) as e:
        mpk.plan(dA, mpk.build_levels(dA, 0), p_max=2)
    assert e.value.status == mpk.MPK_ERR_UNSUPPORTED
    # float64 storage takes the same values
    mpk.plan(mpk.CsrMatrix.from_host(A2, is_symmetric=True), None, p_max=2)

"""Pins for the CPU oracle against facts the paper and mathematics fix.

Each group below targets a plausible oracle mistake: a dropped term or transposed
operand (dense brute force on a non-symmetric integer matrix), a wrong sign or scale
(closed-form eigenpairs), an off-by-one power (permutation powers), a wrong level rule
(Fig. 1, grid closed forms, symmetrisation), a wrong traversal (Fig. 2).
"""
import math

import numpy as np
import pytest

import gen
import oracle
from conftest import read_golden


# ----------------------------------------------------------------------------- SpMV / MPK
def _dense_int_powers(A, x, p):
    """Exact A^k x with Python integers (values and x are integers)."""
    D = [[0] * A.n for _ in range(A.n)]
    for i in range(A.n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            D[i][A.col[e]] += int(A.val[e])
    out = [list(map(int, x))]
    for _ in range(p):
        prev = out[-1]
        out.append([sum(D[i][j] * prev[j] for j in range(A.n)) for i in range(A.n)])
    return out


@pytest.mark.parametrize("n,per_row,p,stream", [(1, 1, 3, 11), (7, 3, 5, 12), (40, 4, 6, 13), (64, 2, 8, 14)])
def test_mpk_dense_bruteforce_exact(n, per_row, p, stream):
    A = gen.random_int_matrix(n, per_row, stream)
    D = A.to_dense()
    assert n == 1 or not np.array_equal(D, D.T)  # non-symmetric: catches A vs A^T
    x = (gen.splitmix64(gen.derive_seed(stream + 100), n) % np.uint64(7)).astype(np.int64) - 3
    Y = oracle.mpk(A, x.astype(np.float64), p)
    ref = _dense_int_powers(A, x, p)
    for k in range(p + 1):
        assert np.array_equal(Y[k, :, 0], np.array(ref[k], dtype=np.float64)), k


def test_mpk_multiple_rhs_columns_independent():
    A = gen.random_int_matrix(30, 3, 21)
    X = (gen.splitmix64(gen.derive_seed(22), 30 * 3) % np.uint64(5)).astype(np.float64).reshape(30, 3) - 2
    Y = oracle.mpk(A, X, 4)
    for r in range(3):
        ref = _dense_int_powers(A, X[:, r].astype(np.int64), 4)
        for k in range(5):
            assert np.array_equal(Y[k, :, r], np.array(ref[k], dtype=np.float64))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,j", [(50, 50), (50, 48), (200, 199), (201, 195)])
def test_mpk_eigenpair_1d(n, j):
    # tridiag(-1,2,-1): lambda_j = 2 - 2 cos(j pi/(n+1)), v_j(i) = sin(i j pi/(n+1)), i=1..n.
    # Modes at the top of the spectrum: rounding error in other eigen-directions then grows
    # no faster than the signal, so 1e-13 holds for every power.
    A = gen.laplacian_1d(n)
    th = j * np.pi / (n + 1)
    v = np.sin(np.arange(1, n + 1) * th)
    lam = 2 - 2 * np.cos(th)
    Y = oracle.mpk(A, v, 8)
    for k in range(9):
        assert _rel(Y[k, :, 0], lam**k * v) < 1e-13, k


def test_mpk_eigenpair_2d_3d():
    nx, ny = 13, 9
    A = gen.laplacian_2d(nx, ny)
    a, b = (nx - 1) * np.pi / (nx + 1), ny * np.pi / (ny + 1)
    X, Yc = np.meshgrid(np.arange(1, nx + 1), np.arange(1, ny + 1), indexing="xy")
    v = (np.sin(X * a) * np.sin(Yc * b)).ravel()  # id = x + nx*y
    lam = 4 - 2 * np.cos(a) - 2 * np.cos(b)
    Y = oracle.mpk(A, v, 6)
    for k in range(7):
        assert _rel(Y[k, :, 0], lam**k * v) < 1e-13

    nx, ny, nz = 6, 5, 4
    A = gen.laplacian_3d(nx, ny, nz)
    t = [nx * np.pi / (nx + 1), (ny - 1) * np.pi / (ny + 1), nz * np.pi / (nz + 1)]
    z, y, x = np.meshgrid(np.arange(1, nz + 1), np.arange(1, ny + 1), np.arange(1, nx + 1), indexing="ij")
    v = (np.sin(x * t[0]) * np.sin(y * t[1]) * np.sin(z * t[2])).ravel()
    lam = 6 - 2 * sum(np.cos(tt) for tt in t)
    Y = oracle.mpk(A, v, 8)
    for k in range(9):
        assert _rel(Y[k, :, 0], lam**k * v) < 1e-13


def test_mpk_row_stochastic_exact():
    A = gen.row_stochastic(300, 3, stream=31)
    Y = oracle.mpk(A, np.ones(300), 12)
    assert np.all(Y == 1.0)


def test_mpk_permutation_powers_exact():
    n = 257
    P, pi = gen.permutation_matrix(n, stream=32)
    x = gen.uniform(gen.derive_seed(33), n)
    Y = oracle.mpk(P, x, 7)
    idx = np.arange(n)
    for k in range(8):
        assert np.array_equal(Y[k, :, 0], x[idx])
        idx = idx[pi]  # (P^{k+1} x)[i] = x[pi^{k+1}(i)]


def test_mpk_rounding_bound_vs_longdouble():
    A = gen.laplacian_2d(20, 17)
    x = gen.uniform(gen.derive_seed(34), A.n)
    Y = oracle.mpk(A, x, 8)[:, :, 0]
    Z = oracle.mpk_longdouble(A, x, 8)
    for k in range(9):
        assert _rel(Y[k], Z[k]) < 1e-14


def test_mpk_stored_order_single_rounding():
    # y = 1e16*1 + 1*1 - 1e16*1 in stored order: the second term is lost to rounding;
    # a different order (or exact arithmetic) would return 1.
    A3 = gen.CSR([0, 3, 4, 5], [0, 1, 2, 1, 2], np.array([1e16, 1.0, -1e16, 1.0, 1.0]))
    Y = oracle.mpk(A3, np.array([1.0, 1.0, 1.0]), 1)
    assert Y[1, 0, 0] == 0.0


# ----------------------------------------------------------------------------- levels
def _fig1_matrix():
    edges = read_golden("fig1_graph.txt")
    n = 20
    r = [i for i in range(n)] + [u for u, v in edges] + [v for u, v in edges]
    c = [i for i in range(n)] + [v for u, v in edges] + [u for u, v in edges]
    return gen.from_coo(n, r, c, np.ones(len(r)) * 2.0)


def test_levels_fig1_exact():
    A = _fig1_matrix()
    level_of, perm, iperm, level_ptr = oracle.levels(A, 0)
    assert np.diff(level_ptr).tolist() == [1, 1, 2, 3, 3, 3, 3, 2, 1, 1]
    golden = dict((o, nl) for o, nl in read_golden("fig1_perm.txt"))
    assert [int(iperm[o]) for o in range(20)] == [golden[o] for o in range(20)]
    assert np.array_equal(perm[iperm], np.arange(20))


@pytest.mark.parametrize("dims", [(5, 4, 3), (8, 8, 8), (1, 9, 2)])
def test_levels_grid_closed_form(dims):
    nx, ny, nz = dims
    A = gen.laplacian_3d(nx, ny, nz)
    level_of, perm, iperm, level_ptr = oracle.levels(A, 0)
    i = np.arange(A.n)
    assert np.array_equal(level_of, i % nx + (i // nx) % ny + i // (nx * ny))
    # inside a level, ascending original index
    for l in range(level_ptr.size - 1):
        seg = perm[level_ptr[l]:level_ptr[l + 1]]
        assert np.all(np.diff(seg) > 0)


def test_levels_chain_is_index():
    A = gen.laplacian_1d(33)
    level_of, perm, _, level_ptr = oracle.levels(A, 0)
    assert np.array_equal(level_of, np.arange(33))
    level_of, _, _, _ = oracle.levels(A, 10)
    assert np.array_equal(level_of, np.abs(np.arange(33) - 10))


def test_levels_symmetrised_pattern():
    # rows 1..n-1 reference column 0 only: edges exist in A's pattern one way only.
    # On A + A^T every vertex neighbours 0, so there are two levels.
    n = 9
    r = list(range(n)) + list(range(1, n))
    c = list(range(n)) + [0] * (n - 1)
    A = gen.from_coo(n, r, c, np.ones(len(r)))
    level_of, _, _, level_ptr = oracle.levels(A, 0)
    assert np.diff(level_ptr).tolist() == [1, n - 1]
    At = gen.from_coo(n, c, r, np.ones(len(r)))
    assert np.array_equal(oracle.levels(At, 0)[0], level_of)


def test_levels_disconnected_restart():
    # components {0,1,2} (chain) and {3,4} (edge) and {5} (isolated)
    n = 6
    e = [(0, 1), (1, 2), (3, 4)]
    r = list(range(n)) + [u for u, v in e] + [v for u, v in e]
    c = list(range(n)) + [v for u, v in e] + [u for u, v in e]
    A = gen.from_coo(n, r, c, np.ones(len(r)))
    level_of, perm, _, level_ptr = oracle.levels(A, 0)
    assert level_of.tolist() == [0, 1, 2, 3, 4, 5]
    level_of, perm, _, level_ptr = oracle.levels(A, 4)
    # from 4: L0={4}, L1={3}, restart at 0: L2={0}, L3={1}, L4={2}, restart at 5: L5={5}
    assert level_of.tolist() == [2, 3, 4, 1, 0, 5]


def test_levels_adjacency_invariant_random():
    # Sec. 3: neighbours of L(i) lie in L(i-1), L(i), L(i+1)
    for s, n in [(41, 500), (42, 3000)]:
        A = gen.banded_random(n, stream=s)
        level_of, perm, iperm, level_ptr = oracle.levels(A, 0)
        rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
        assert np.max(np.abs(level_of[rows] - level_of[A.col])) <= 1
        assert np.array_equal(np.sort(perm), np.arange(n))


# ----------------------------------------------------------------------------- permutation
def test_permute_is_pap_with_stored_order():
    A = gen.random_int_matrix(25, 4, 51)
    level_of, perm, iperm, _ = oracle.levels(A, 3)
    prp, pci, pva = oracle.permute(A, perm, iperm)
    D = A.to_dense()
    Pd = gen.CSR(prp, pci, pva).to_dense()
    assert np.array_equal(Pd, D[np.ix_(perm, perm)])
    for r in range(25):
        old = perm[r]
        seg_old = slice(A.row_ptr[old], A.row_ptr[old + 1])
        seg_new = slice(prp[r], prp[r + 1])
        assert np.array_equal(pci[seg_new], iperm[A.col[seg_old]])
        assert np.array_equal(pva[seg_new], A.val[seg_old])


# ----------------------------------------------------------------------------- groups
def test_groups_equal_levels():
    # 12 levels of 10 rows with 3 entries each: bytes(level) = 12*30 + 4*10 + 16*10 = 560
    L, rows, per = 12, 10, 3
    level_ptr = np.arange(L + 1, dtype=np.int32) * rows
    rp = np.arange(L * rows + 1, dtype=np.int32) * per
    for k in (1, 2, 3, 5):
        g = oracle.groups(level_ptr, rp, budget=560 * k)
        assert np.array_equal(g, np.array(list(range(0, L, k)) + [L]))
        g = oracle.groups(level_ptr, rp, budget=560 * k + 559)
        assert np.array_equal(g, np.array(list(range(0, L, k)) + [L]))


def test_groups_bulky_singleton_and_cover():
    level_rows = [2, 2, 50, 2, 2, 2]
    level_ptr = np.concatenate([[0], np.cumsum(level_rows)]).astype(np.int32)
    rp = np.arange(level_ptr[-1] + 1, dtype=np.int32) * 2  # 2 entries per row
    per_row = 12 * 2 + 4 + 16
    g = oracle.groups(level_ptr, rp, budget=4 * per_row)
    assert g.tolist() == [0, 2, 3, 5, 6]  # level 2 is bulky and alone
    assert g[0] == 0 and g[-1] == len(level_rows) and np.all(np.diff(g) > 0)
    # m right-hand sides and 4-byte values change the per-row cost
    g2 = oracle.groups(level_ptr, rp, budget=4 * (8 * 2 + 4 + 32), val_bytes=4, m=2)
    assert g2.tolist() == [0, 2, 3, 5, 6]


# ----------------------------------------------------------------------------- schedule
def test_lp_labels_fig2():
    golden = np.array(read_golden("fig2_lp_labels.txt"))
    assert np.array_equal(oracle.lp_labels(10, 5), golden)
    assert np.array_equal(oracle.lp_labels(10, 5, skew=1), golden)
    # Sec. 3 text: L(5) at p=1 runs at step 15 and is reused at step 21 (p=2), p_m+1 steps later
    lab = oracle.lp_labels(10, 5)
    assert lab[0, 5] == 15 and lab[1, 5] == 21


@pytest.mark.parametrize("skew", [1, 2, 3, 4])
def test_lp_order_respects_dependencies(skew):
    # every cell runs after (i-1, p-1), (i, p-1) and (i+1, p-1), the Sec. 3 dependency rule
    L, pm = 13, 6
    lab = oracle.lp_labels(L, pm, skew)
    assert sorted(lab.ravel().tolist()) == list(range(L * pm))
    for p in range(1, pm):
        for i in range(L):
            for j in (i - 1, i, i + 1):
                if 0 <= j < L:
                    assert lab[p, i] > lab[p - 1, j]


def test_lp_order_skew_lines_are_independent():
    # with skew >= 2 no cell depends on another cell of its own line g + skew*k
    L, pm = 11, 5
    for skew in (2, 3):
        for p in range(2, pm + 1):
            for i in range(L):
                for j in (i - 1, i, i + 1):
                    if 0 <= j < L:
                        assert (i + skew * p) - (j + skew * (p - 1)) >= skew - 1 >= 1


@pytest.mark.parametrize("skew", [1, 2, 3])
def test_lb_mpk_bitwise_equals_plain(skew):
    A = gen.laplacian_3d(9, 7, 5)
    level_of, perm, iperm, level_ptr = oracle.levels(A, 0)
    prp, pci, pva = oracle.permute(A, perm, iperm)
    X = gen.vector(A.n, 2, stream=61)
    Yplain = oracle.mpk(A, X, 6)
    for budget in (1, 2000, 10**9):
        gl = oracle.groups(level_ptr, prp, budget, m=2)
        group_rows = level_ptr[gl]
        Ylb = oracle.lb_mpk(prp, pci, pva, X[perm], 6, group_rows, skew=skew)
        assert np.array_equal(Ylb[:, iperm, :], Yplain)


def test_lb_mpk_detects_a_wrong_order():
    # planted mistake: skew 0 runs all powers of a group before the next group, so (g, 2)
    # reads group g+1 at power 1 before it exists; the run must not match back-to-back SpMV
    A = gen.laplacian_3d(9, 7, 5)
    level_of, perm, iperm, level_ptr = oracle.levels(A, 0)
    prp, pci, pva = oracle.permute(A, perm, iperm)
    X = gen.vector(A.n, 1, stream=62)
    gl = oracle.groups(level_ptr, prp, 1)
    Ybad = oracle.lb_mpk(prp, pci, pva, X[perm], 3, level_ptr[gl], skew=0)
    assert np.isnan(Ybad[2:]).any()
    lab = oracle.lp_labels(10, 3, skew=0)
    assert lab[1, 4] < lab[0, 5]  # (i=4, p=2) before (i=5, p=1): the rule is broken


# ----------------------------------------------------------------------------- Chebyshev
def test_cheb_eigenvector_single_terms():
    n = 60
    A = gen.laplacian_1d(n)
    lo, hi = gen.gershgorin_bounds(A)  # [0, 4]
    assert (lo, hi) == (0.0, 4.0)
    scale, shift = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    j = 7
    th = j * np.pi / (n + 1)
    v = np.sin(np.arange(1, n + 1) * th)
    lamp = (2 - 2 * np.cos(th) - shift) / scale
    for k in (0, 1, 2, 5, 16):
        c = np.zeros(k + 1)
        c[k] = 1.0
        out = oracle.cheb(A, v, k, c, scale=scale, shift=shift)[:, 0]
        assert _rel(out, np.cos(k * np.arccos(lamp)) * v) < 1e-12, k


def test_bessel_against_published_and_scipy():
    J = oracle.bessel_j(5, 1.0)
    assert abs(J[0] - 0.7651976865579666) < 1e-15   # Abramowitz & Stegun Table 9.1
    assert abs(J[1] - 0.4400505857449335) < 1e-15
    J10 = oracle.bessel_j(30, 10.0)
    assert abs(J10[0] - (-0.2459357644513483)) < 1e-14
    assert abs(J10[1] - 0.04347274616886144) < 1e-14
    assert abs(J10[0] ** 2 + 2 * np.sum(J10[1:] ** 2) - 1.0) < 1e-13
    sp = pytest.importorskip("scipy.special")
    for x in (0.5, 3.0, 25.0):
        J = oracle.bessel_j(60, x)
        assert np.max(np.abs(J - sp.jv(np.arange(61), x))) < 1e-14


def test_cheb_time_step_matches_exponential():
    # Sec. 7: exp(-i dt H) v = e^{-i dt c}[J0(a dt) v0 + 2 sum (-i)^k J_k(a dt) v_k] with H = a H' + c
    n = 40
    A = gen.laplacian_1d(n)
    lo, hi = gen.gershgorin_bounds(A)
    a, c = (hi - lo) / 2 * 1.01, (hi + lo) / 2
    dt, M = 2.0, 40
    J = oracle.bessel_j(M, a * dt)
    coef = np.array([J[0]] + [2 * (-1j) ** k * J[k] for k in range(1, M + 1)]) * np.exp(-1j * dt * c)
    j = 5
    th = j * np.pi / (n + 1)
    v = np.sin(np.arange(1, n + 1) * th)
    lam = 2 - 2 * np.cos(th)
    psi = np.stack([v, np.zeros(n)], axis=1)  # complex state as (re, im) columns
    out = oracle.cheb(A, psi, M, coef.real.copy(), coef.imag.copy(), scale=a, shift=c)
    got = out[:, 0] + 1j * out[:, 1]
    want = np.exp(-1j * dt * lam) * v
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12


# ----------------------------------------------------------------------------- binary32 accumulation
def test_mpk_acc32_exact_when_every_sum_fits_binary32():
    # small integers: every product, partial sum and power is an integer below 2^24, so the
    # binary32 row sums are exact and equal the binary64 oracle and exact integer arithmetic
    A = gen.random_int_matrix(40, 3, 31)
    x = (gen.splitmix64(gen.derive_seed(131), 40 * 2) % np.uint64(5)).astype(np.float64).reshape(40, 2) - 2
    Y32 = oracle.mpk_acc32(A, x, 5)
    assert np.abs(Y32).max() < 2 ** 24
    assert np.array_equal(Y32.view(np.uint64), oracle.mpk(A, x, 5).view(np.uint64))
    for r in range(2):
        ref = _dense_int_powers(A, x[:, r].astype(np.int64), 5)
        for k in range(6):
            assert np.array_equal(Y32[k, :, r], np.array(ref[k], dtype=np.float64))


def test_mpk_acc32_rounds_input_sum_and_product_once():
    # hand-computed binary32 cases, u = 2^-24:
    # (a) the input is rounded: x = 1 + 2^-30 -> 1.0f, so 3 x -> 3 exactly (binary64 keeps 3 + 3*2^-30);
    A = gen.CSR([0, 1], [0], np.array([3.0]))
    assert oracle.mpk_acc32(A, np.array([1 + 2.0 ** -30]), 1)[1, 0, 0] == 3.0
    assert oracle.mpk(A, np.array([1 + 2.0 ** -30]), 1)[1, 0, 0] == 3 + 3 * 2.0 ** -30
    # (b) the sum is rounded: 1 + 2^-24 is a tie between 1 and 1 + 2^-23 -> 1.0f (even);
    A = gen.CSR([0, 2, 3], [0, 1, 1], np.array([1.0, 1.0, 1.0]))
    y = oracle.mpk_acc32(A, np.array([1.0, 2.0 ** -24]), 1)[1, :, 0]
    assert y[0] == 1.0 and y[1] == 2.0 ** -24
    # (c) product and sum are rounded once (fmaf): stored order (-1, then a), a = x0 = 1 + 2^-12:
    #     fmaf(a, x0, -1) = 2^-11 + 2^-24 exactly, while a rounded product gives 2^-11
    a = 1 + 2.0 ** -12
    A = gen.CSR([0, 2, 3], [1, 0, 1], np.array([-1.0, a, 1.0]))
    y = oracle.mpk_acc32(A, np.array([a, 1.0]), 1)[1, :, 0]
    assert y[0] == 2.0 ** -11 + 2.0 ** -24
    # values that binary32 cannot hold are refused
    with pytest.raises(RuntimeError):
        oracle.mpk_acc32(gen.CSR([0, 1], [0], np.array([0.1])), np.array([1.0]), 1)


def test_mpk_acc32_elementwise_error_bound():
    # each power is the binary32 evaluation of A times the binary32 rounding of the previous
    # power: |y_k - A fl32(y_{k-1})| <= gamma_w (|A| |fl32(y_{k-1})|) row by row, gamma_w = w u / (1 - w u)
    # with w the row's entry count and u = 2^-24 (the standard bound for a recursive fma sum)
    A = gen.banded_random(500, stream=132)
    vals = A.val.astype(np.float32).astype(np.float64)
    A = gen.CSR(A.row_ptr, A.col, vals)
    X = gen.vector(A.n, 1, stream=133)
    Y = oracle.mpk_acc32(A, X, 6)
    D = A.to_dense().astype(np.longdouble)
    w = np.diff(A.row_ptr).astype(np.longdouble)
    u = np.longdouble(2.0) ** -24
    gamma = w * u / (1 - w * u)
    err_total = 0.0
    for k in range(1, 7):
        xin = Y[k - 1, :, 0].astype(np.float32).astype(np.longdouble)
        exact = D @ xin
        bound = gamma * (np.abs(D) @ np.abs(xin))
        diff = np.abs(Y[k, :, 0].astype(np.longdouble) - exact)
        assert np.all(diff <= bound), k
        err_total += float(np.sum(diff))
    assert err_total > 0  # the binary32 path really rounds


def test_cheb_acc32_integer_case_equals_binary64():
    # scale 1, shift 0 and small integers: A' = A, every w and every recurrence value is an
    # integer below 2^24, so the binary32 products are exact and the two oracles agree
    A = gen.random_int_matrix(25, 2, 34)
    x = (gen.splitmix64(gen.derive_seed(134), 25 * 2) % np.uint64(3)).astype(np.float64).reshape(25, 2) - 1
    c = np.array([1.0, -2.0, 0.5, 3.0, 1.0, -1.0])
    want = oracle.cheb(A, x, 5, c, scale=1.0, shift=0.0)
    got = oracle.cheb_acc32(A, x, 5, c, scale=1.0, shift=0.0)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_cheb_acc32_keeps_the_recurrence_in_binary64():
    # 1 x 1 matrix [2], x = 1 + 2^-30, scale 1, shift 0: w = 2 * fl32(x) = 2, then
    # v_1 = fma(1, 2, 0 * x) = 2, v_2 = fma(2, 2 * fl32(v_1) = 4, fma(0, v_1, -x)) = 8 - x,
    # which keeps x's low bits (a binary32 recurrence would lose them)
    A = gen.CSR([0, 1], [0], np.array([2.0]))
    x = 1 + 2.0 ** -30
    got = oracle.cheb_acc32(A, np.array([x]), 2, np.array([0.0, 0.0, 1.0]), scale=1.0, shift=0.0)
    assert got[0, 0] == 8 - x


def test_parallel_oracle_leg_is_the_same_computation():
    # the row-parallel timing leg of the CPU baseline runs the serial row body on several
    # threads: the same bits as the serial oracle
    A = gen.banded_random(3000, stream=135)
    X = gen.vector(A.n, 2, stream=136)
    Y, threads = oracle.mpk_parallel(A, X, 5)
    assert threads >= 1
    assert np.array_equal(Y.view(np.uint64), oracle.mpk(A, X, 5).view(np.uint64))


def test_load_sum_reads_every_element_once():
    # the host load-bandwidth kernel of the CPU baseline: an exact sum (integers, any thread
    # split), so a skipped or repeated chunk of the buffer changes the result
    buf = np.arange(1, 100001, dtype=np.float64)
    assert oracle.load_sum(buf, 1) == 100000 * 100001 / 2
    assert oracle.load_sum(buf, 3) == 3 * 100000 * 100001 / 2
    assert oracle.load_sum(buf[:0], 2) == 0.0
    assert oracle.load_bandwidth(1 << 22, 2) > 0


# ----------------------------------------------------------------------------- bulky levels split
def _star(k=4):
    # row 0 joined to rows 1..k, every row with a diagonal: levels {0}, {1..k}
    r = list(range(k + 1)) + [0] * k + list(range(1, k + 1))
    c = list(range(k + 1)) + list(range(1, k + 1)) + [0] * k
    return gen.from_coo(k + 1, r, c, np.linspace(1.0, 2.0, len(r)))


def test_groups_split_hand_computed():
    # row bytes (8 + 4) nnz + 4 + 16: row 0 (5 entries) 80, rows 1..4 (2 entries) 44; levels 80 and 176
    A = _star()
    lo, pe, ip, lp = oracle.levels(A, 0)
    prp, _, _ = oracle.permute(A, pe, ip)
    assert oracle.groups_split(lp, prp, 100).tolist() == [0, 1, 3, 5]   # {0} | {1,2} 88 | {3,4} 88
    assert oracle.groups_split(lp, prp, 200).tolist() == [0, 1, 5]      # 80 + 176 > 200, 176 fits
    assert oracle.groups_split(lp, prp, 300).tolist() == [0, 5]         # both levels in one group
    assert oracle.groups_split(lp, prp, 50).tolist() == [0, 1, 2, 3, 4, 5]  # single rows over budget


@pytest.mark.parametrize("budget", [2000, 20000, 60000])
def test_groups_split_invariants(budget):
    A = gen.laplacian_3d(14, 11, 9)
    lo, pe, ip, lp = oracle.levels(A, 0)
    prp, _, _ = oracle.permute(A, pe, ip)
    gr = oracle.groups_split(lp, prp, budget)
    rb = 12 * np.diff(prp) + 4 + 16
    assert gr[0] == 0 and gr[-1] == A.n and np.all(np.diff(gr) > 0)
    lev = np.searchsorted(lp, np.arange(A.n), side="right") - 1
    for g in range(gr.size - 1):
        rows = np.arange(gr[g], gr[g + 1])
        ls = np.unique(lev[rows])
        lvl_bytes = [rb[lp[l]:lp[l + 1]].sum() for l in ls]
        if any(b > budget for b in lvl_bytes):   # a piece of a bulky level: one level, within budget
            assert ls.size == 1 and (rb[rows].sum() <= budget or rows.size == 1)
        else:                                     # whole levels, within budget
            assert gr[g] in lp and gr[g + 1] in lp
            assert rb[rows].sum() <= budget
    # without bulky levels the rule is orc_groups'
    big = 10 ** 9
    assert np.array_equal(oracle.groups_split(lp, prp, big), lp[oracle.groups(lp, prp, big)])


@pytest.mark.parametrize("budget", [50, 100, 2000, 20000])
def test_wave_order_is_exact_where_lines_read_early(budget):
    # split groups break the +-1 rule of levels; the wave order still gives back-to-back SpMV bit
    # for bit, while the fixed line order g + 3k reads unfinished (NaN) inputs on the star
    for A in (_star(6), gen.laplacian_3d(9, 8, 7), gen.banded_random(400, stream=140)):
        lo, pe, ip, lp = oracle.levels(A, 0)
        prp, pci, pva = oracle.permute(A, pe, ip)
        gr = oracle.groups_split(lp, prp, budget)
        X = gen.vector(A.n, 2, stream=141)[pe]
        want = oracle.mpk(gen.CSR(prp, pci, pva), X, 6)
        got = oracle.lb_mpk_waves(prp, pci, pva, X, 6, gr)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    A = _star(6)
    lo, pe, ip, lp = oracle.levels(A, 0)
    prp, pci, pva = oracle.permute(A, pe, ip)
    gr = oracle.groups_split(lp, prp, 50)
    assert np.isnan(oracle.lb_mpk(prp, pci, pva, np.ones(A.n), 3, gr, skew=3)).any()

"""Pins for the seeded input generators: closed-form sizes from the paper and textbook facts."""
import math

import numpy as np
import pytest

import gen
from conftest import read_golden


def test_table5_closed_form_and_crs_size():
    # Table 5: nnz of an open-boundary 7-point lattice is 7n - 2(LxLy + LyLz + LxLz) and the
    # CRS size is (4 N_r + 12 N_nz) bytes (Sec. 6, benchmark matrices).
    for lx, ly, lz, nr, nnz, mib in read_golden("table5_anderson.txt"):
        n = lx * ly * lz
        assert n == nr
        assert 7 * n - 2 * (lx * ly + ly * lz + lx * lz) == nnz
        assert round((4 * nr + 12 * nnz) / 2**20) == mib


def test_table5_first_row_generated():
    A = gen.laplacian_3d(160, 160, 160)
    assert (A.n, A.nnz) == (4096000, 28518400)
    assert round(A.crs_bytes() / 2**20) == 342


@pytest.mark.parametrize("dims", [(3, 4, 5), (7, 2, 9), (1, 1, 6), (16, 16, 16)])
def test_laplacian_3d_structure(dims):
    nx, ny, nz = dims
    A = gen.laplacian_3d(nx, ny, nz)
    n = nx * ny * nz
    assert A.nnz == 7 * n - 2 * (nx * ny + ny * nz + nx * nz)
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) == 6)
    # every off-diagonal entry is -1 and joins grid points at Manhattan distance 1
    r, c = np.nonzero(D - np.diag(np.diag(D)))
    assert np.all(D[r, c] == -1)
    coord = lambda i: np.stack([i % nx, (i // nx) % ny, i // (nx * ny)])
    assert np.all(np.abs(coord(r) - coord(c)).sum(axis=0) == 1)
    for i in range(n):  # columns ascending inside each row
        assert np.all(np.diff(A.col[A.row_ptr[i]:A.row_ptr[i + 1]]) > 0)


def test_headline_sizes_closed_form():
    n = 256**3
    assert n == 16_777_216
    assert 7 * n - 2 * 3 * 256 * 256 == 117_047_296


def test_laplacian_2d_small_config():
    A, p = gen.config_small()
    assert (A.n, A.nnz, p) == (4096, 20224, 4)
    assert A.nnz == 5 * 4096 - 2 * (64 + 64)


@pytest.mark.parametrize("s", [2, 3, 5, 11])
def test_stencil27_count(s):
    assert gen.stencil27(s).nnz == (3 * s - 2) ** 3


def test_xxz_sector_size_and_structure():
    L = 10
    A = gen.xxz_chain(L, stream=4)
    assert A.n == math.comb(L, L // 2)
    D = A.to_dense()
    assert np.allclose(D, D.T)
    off = D - np.diag(np.diag(D))
    assert set(np.unique(off[off != 0])) == {0.5}
    # each basis state connects to one state per anti-aligned bond (periodic chain)
    basis = gen.xxz_basis(L)
    for i in range(A.n):
        s = int(basis[i])
        anti = sum(((s >> b) & 1) != ((s >> ((b + 1) % L)) & 1) for b in range(L))
        assert np.count_nonzero(off[i]) == anti
    assert math.comb(24, 12) == 2_704_156


def test_splitmix64_reference_values():
    # splitmix64 from seed 0: first outputs published with the algorithm (Vigna's reference code)
    u = gen.splitmix64(0, 3)
    assert [hex(int(v)) for v in u] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4", "0x6c45d188009454f"]


def test_uniform_range_and_determinism():
    a = gen.uniform(gen.derive_seed(1), 100000)
    b = gen.uniform(gen.derive_seed(1), 100000)
    assert np.array_equal(a, b)
    assert a.min() >= -1.0 and a.max() < 1.0
    assert abs(a.mean()) < 0.01


def test_row_stochastic_and_permutation_generators():
    A = gen.row_stochastic(50, 3, stream=5)
    assert np.all(np.diff(A.row_ptr) == 8)
    assert np.all(A.val == 0.125)
    P, pi = gen.permutation_matrix(40, stream=6)
    assert sorted(pi.tolist()) == list(range(40))
    assert np.array_equal(P.col, pi)


def test_banded_random_shape():
    n = 20000
    A = gen.banded_random(n, stream=7)
    D_bw = np.max(np.abs(np.repeat(np.arange(n), np.diff(A.row_ptr)) - A.col))
    assert D_bw <= math.ceil(n / 100)
    assert 12 < A.nnz / n < 16

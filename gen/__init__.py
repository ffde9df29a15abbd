"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

This module only *builds inputs*: CSR matrices shaped like the paper's workloads and
dense vectors drawn from a counter-based generator.  It contains none of the matrix
power kernel's arithmetic (no SpMV, no BFS, no grouping), so both the oracle and the
CUDA path can consume it without sharing any of the method's code.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used in counter mode: element i of
stream s is mix(s + (i+1) * 0x9E3779B97F4A7C15).  Uniform[-1,1) doubles take the top
53 bits; normals use the Box-Muller transform.

CSR convention everywhere: int32 row pointers (n+1) and column indices, column indices
ascending inside every row, float64 values.
"""
from __future__ import annotations

import math
import numpy as np

BASE_SEED = 20240520
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ----------------------------------------------------------------------------- PRNG
def derive_seed(stream: int, base: int = BASE_SEED) -> int:
    """One independent splitmix64 stream per matrix or vector, named by an integer."""
    z = (base * 0x9E3779B97F4A7C15 + (stream + 1) * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF
    return int(_mix64_scalar(z))


def _mix64_scalar(z: int) -> int:
    z &= 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Elements offset..offset+count-1 of the splitmix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """float64 in [lo, hi): (u >> 11) * 2^-53 mapped affinely."""
    u = (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on two uniform (0,1] streams."""
    m = (count + 1) // 2
    u1 = ((splitmix64(seed, m) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (splitmix64(seed, m, offset=m) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


def vector(n: int, nrhs: int = 1, stream: int = 1) -> np.ndarray:
    """A dense block X (n x nrhs, row-major) with entries uniform in [-1,1)."""
    return uniform(derive_seed(stream), n * nrhs).reshape(n, nrhs)


# ----------------------------------------------------------------------------- CSR helpers
class CSR:
    """Host CSR matrix: row_ptr/col int32, val float64 (or float32)."""

    def __init__(self, row_ptr, col, val, name=""):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def crs_bytes(self, val_bytes: int = 8) -> int:
        """CRS storage as the paper counts it: 4 B per row pointer, 4+val_bytes per entry."""
        return 4 * self.n + (4 + val_bytes) * self.nnz

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col), self.val.astype(np.float64))
        return d

    def with_values(self, val) -> "CSR":
        return CSR(self.row_ptr, self.col, val, self.name)


def from_coo(n: int, rows, cols, vals, name="", sum_duplicates=True) -> CSR:
    """Sort COO triples by (row, col) and compress; duplicates are summed."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    if sum_duplicates and key.size:
        uniq, start = np.unique(key, return_index=True)
        vals = np.add.reduceat(vals, start)
        key = uniq
    r = key // n
    c = key - r * n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(row_ptr, c, vals, name)


def _stencil(dims, offsets, diag_val, off_val, name) -> CSR:
    """Constant-coefficient stencil on a lexicographic grid with open (Dirichlet) boundaries.

    dims = (nx, ny, nz); id = x + nx*(y + ny*z).  `offsets` is a list of (dx,dy,dz)
    including (0,0,0); entries come out sorted by column because offsets are sorted by
    their linear displacement.
    """
    nx, ny, nz = dims
    n = nx * ny * nz
    offs = sorted(offsets, key=lambda o: o[0] + nx * (o[1] + ny * o[2]))
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    cnt = np.zeros(n, dtype=np.int64)
    masks = []
    for dx, dy, dz in offs:
        m = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & (z + dz >= 0) & (z + dz < nz)
        masks.append(m)
        cnt += m
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    pos = row_ptr[:-1].copy()
    for (dx, dy, dz), m in zip(offs, masks):
        d = dx + nx * (dy + ny * dz)
        rows = idx[m]
        p = pos[m]
        col[p] = (rows + d).astype(np.int32)
        val[p] = diag_val if (dx, dy, dz) == (0, 0, 0) else off_val
        pos[m] += 1
    del masks
    return CSR(row_ptr, col, val, name)


# ----------------------------------------------------------------------------- workloads
def laplacian_1d(n: int) -> CSR:
    """tridiag(-1, 2, -1), Dirichlet."""
    return _stencil((n, 1, 1), [(-1, 0, 0), (0, 0, 0), (1, 0, 0)], 2.0, -1.0, f"lap1d_{n}")


def laplacian_2d(nx: int, ny: int) -> CSR:
    """5-point Laplacian, values {4 diag, -1}, Dirichlet, lexicographic (id = x + nx*y)."""
    offs = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    return _stencil((nx, ny, 1), offs, 4.0, -1.0, f"lap2d_{nx}x{ny}")


def laplacian_3d(nx: int, ny: int, nz: int) -> CSR:
    """7-point Laplacian, values {6 diag, -1}, open boundaries, lexicographic."""
    offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    return _stencil((nx, ny, nz), offs, 6.0, -1.0, f"lap3d_{nx}x{ny}x{nz}")


def stencil27(s: int) -> CSR:
    """27-point stencil on an s^3 grid, values {26 diag, -1}, open boundaries."""
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return _stencil((s, s, s), offs, 26.0, -1.0, f"st27_{s}")


def banded_random(n: int, stream: int, per_row: int = 7, band_frac: float = 0.01) -> CSR:
    """Random symmetric banded graph: `per_row` upper entries per row drawn uniformly in
    (i, i + ceil(n*band_frac)], mirrored, plus the diagonal; duplicates merged (summed);
    values N(0,1), symmetric."""
    bw = max(1, math.ceil(n * band_frac))
    seed = derive_seed(stream)
    u = splitmix64(seed, n * per_row)
    off = (u % np.uint64(bw)).astype(np.int64) + 1
    rows = np.repeat(np.arange(n, dtype=np.int64), per_row)
    cols = rows + off
    keep = cols < n
    rows, cols = rows[keep], cols[keep]
    v = normal(derive_seed(stream + 1000), rows.size)
    d = normal(derive_seed(stream + 2000), n)
    r_all = np.concatenate([rows, cols, np.arange(n)])
    c_all = np.concatenate([cols, rows, np.arange(n)])
    v_all = np.concatenate([v, v, d])
    return from_coo(n, r_all, c_all, v_all, name=f"band_{n}")


def xxz_basis(L: int) -> np.ndarray:
    """All L-bit patterns with L/2 bits set (the Sz=0 sector), ascending."""
    states = np.arange(1 << L, dtype=np.int64)
    pc = np.zeros_like(states)
    t = states.copy()
    for _ in range(L):
        pc += t & 1
        t >>= 1
    return states[pc == L // 2]


def xxz_chain(L: int = 24, stream: int = 4, jxy: float = 1.0, jz: float = 0.5) -> CSR:
    """Spin-1/2 XXZ chain, periodic, Sz=0 sector:
    H = sum_i [ jxy/2 (S+_i S-_{i+1} + h.c.) + jz Sz_i Sz_{i+1} ] + sum_i h_i Sz_i,
    h_i ~ U[-1,1] from the seeded stream.  Off-diagonal entries are jxy/2."""
    basis = xxz_basis(L)
    n = basis.size
    h = uniform(derive_seed(stream), L)
    diag = np.zeros(n)
    rows, cols = [np.arange(n)], []
    offr, offc = [], []
    for i in range(L):
        j = (i + 1) % L
        bi = (basis >> i) & 1
        bj = (basis >> j) & 1
        szi, szj = bi - 0.5, bj - 0.5
        diag += jz * szi * szj + h[i] * szi
        flip = bi != bj
        src = np.nonzero(flip)[0]
        dst_state = basis[src] ^ ((1 << i) | (1 << j))
        offr.append(src)
        offc.append(np.searchsorted(basis, dst_state))
    r = np.concatenate([np.arange(n)] + offr)
    c = np.concatenate([np.arange(n)] + offc)
    v = np.concatenate([diag, np.full(sum(a.size for a in offr), jxy / 2)])
    return from_coo(n, r, c, v, name=f"xxz_{L}", sum_duplicates=True)


def row_stochastic(n: int, log2_per_row: int, stream: int) -> CSR:
    """Every row holds 2^m distinct columns of value 2^-m, so A^k 1 = 1 exactly."""
    k = 1 << log2_per_row
    assert k <= n
    seed = derive_seed(stream)
    cols = np.empty((n, k), dtype=np.int64)
    u = splitmix64(seed, n * 4 * k).reshape(n, 4 * k) % np.uint64(n)
    for i in range(n):
        seen = []
        for c in u[i]:
            c = int(c)
            if c not in seen:
                seen.append(c)
            if len(seen) == k:
                break
        j = 0
        while len(seen) < k:
            if j not in seen:
                seen.append(j)
            j += 1
        cols[i] = sorted(seen)
    rows = np.repeat(np.arange(n), k)
    return from_coo(n, rows, cols.ravel(), np.full(n * k, 2.0 ** -log2_per_row), name="stoch")


def permutation_matrix(n: int, stream: int):
    """A = P with P[i, pi[i]] = 1; returns (CSR, pi)."""
    pi = np.argsort(splitmix64(derive_seed(stream), n), kind="stable").astype(np.int64)
    return from_coo(n, np.arange(n), pi, np.ones(n), name="perm"), pi


def random_int_matrix(n: int, per_row: int, stream: int, lo: int = -3, hi: int = 3) -> CSR:
    """Small non-symmetric integer matrix (for exact dense brute-force checks)."""
    seed = derive_seed(stream)
    u = splitmix64(seed, n * per_row * 2)
    cols = (u[: n * per_row] % np.uint64(n)).astype(np.int64)
    vals = (u[n * per_row:] % np.uint64(hi - lo + 1)).astype(np.int64) + lo
    rows = np.repeat(np.arange(n), per_row)
    return from_coo(n, rows, cols, vals.astype(np.float64), name="int", sum_duplicates=True)


def gershgorin_bounds(A: CSR):
    """Guaranteed spectral enclosure [lo, hi] from Gershgorin discs (inputs for Chebyshev scaling)."""
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    v = A.val.astype(np.float64)
    d = np.zeros(A.n)
    is_d = rows == A.col
    np.add.at(d, rows[is_d], v[is_d])
    r = np.zeros(A.n)
    np.add.at(r, rows[~is_d], np.abs(v[~is_d]))
    return float(np.min(d - r)), float(np.max(d + r))


# ----------------------------------------------------------------------------- named configs
def config_small():
    """2-D 5-point Laplacian on 64x64 (n=4096, 20,224 nnz), x ~ U[-1,1), p=4."""
    return laplacian_2d(64, 64), 4


def config_headline(side: int = 256):
    """3-D 7-point Laplacian on side^3 (256^3: n=16,777,216, nnz=117,047,296), p=8."""
    return laplacian_3d(side, side, side), 8

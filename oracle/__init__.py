"""CPU oracle for the level-blocked matrix power kernel.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by the
cpu_baseline / reference legs of bench.py, never by the product package.  The C
source (oracle.c) is plain serial code that follows the paper step by step; this
module only compiles it (gcc, -ffp-contract=off) and marshals numpy arrays.

Every function returns numpy arrays and raises on a non-zero status.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        # the row-parallel timing leg uses OpenMP where the compiler has it (same arithmetic either way)
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
            lib.orc_mpk.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, i32, _f64p]
            lib.orc_mpk_longdouble.argtypes = [i32, _i32p, _i32p, _f64p, _f64p, i32, _f64p]
            lib.orc_levels.argtypes = [i32, _i32p, _i32p, i32, _i32p, _i32p, _i32p, _i32p, C.POINTER(i32)]
            lib.orc_permute.argtypes = [i32, _i32p, _i32p, _f64p, _i32p, _i32p, _i32p, _i32p, _f64p]
            lib.orc_groups.argtypes = [i32, _i32p, _i32p, i32, i32, i64, _i32p, C.POINTER(i32)]
            lib.orc_lp_labels.argtypes = [i32, i32, i32, _i32p]
            lib.orc_lb_mpk.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, i32, i32, _i32p, i32, _f64p]
            lib.orc_cheb.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, i32, _f64p, C.c_void_p,
                                     f64, f64, _f64p]
            lib.orc_bessel_j.argtypes = [i32, f64, _f64p]
            lib.orc_mpk_acc32.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, i32, _f64p]
            lib.orc_cheb_acc32.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, i32, _f64p, C.c_void_p,
                                           f64, f64, _f64p]
            lib.orc_groups_split.argtypes = [i32, _i32p, _i32p, i32, i32, i64, _i32p, C.POINTER(i32)]
            lib.orc_lb_mpk_waves.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, i32, i32, _i32p, _f64p]
            lib.orc_mpk_omp.argtypes = [i32, _i32p, _i32p, _f64p, i32, _f64p, i32, _f64p, C.POINTER(i32)]
            lib.orc_load_sum.argtypes = [_f64p, i64, i32]
            lib.orc_load_sum.restype = f64
            for f in ("orc_groups_split", "orc_lb_mpk_waves", "orc_mpk", "orc_mpk_omp", "orc_mpk_longdouble", "orc_levels", "orc_permute", "orc_groups",
                      "orc_lp_labels", "orc_lb_mpk", "orc_cheb", "orc_bessel_j", "orc_mpk_acc32",
                      "orc_cheb_acc32"):
                getattr(lib, f).restype = C.c_int
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def _csr(A):
    return (np.ascontiguousarray(A.row_ptr, np.int32), np.ascontiguousarray(A.col, np.int32),
            np.ascontiguousarray(A.val, np.float64))


def _block(X, n):
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X.reshape(n, 1)
    return X


def mpk(A, X, p: int) -> np.ndarray:
    """Y[k] = A^k X for k = 0..p, shape (p+1, n, m); back-to-back SpMV (Sec. 3)."""
    rp, ci, va = _csr(A)
    X = _block(X, A.n)
    m = X.shape[1]
    Y = np.empty((p + 1, A.n, m), dtype=np.float64)
    _check(_L().orc_mpk(A.n, rp, ci, va, m, X, p, Y), "mpk")
    return Y


def mpk_parallel(A, X, p: int):
    """orc_mpk with each power's rows shared out over the host cores (same bits); returns
    (Y, threads used)."""
    rp, ci, va = _csr(A)
    X = _block(X, A.n)
    m = X.shape[1]
    Y = np.empty((p + 1, A.n, m), dtype=np.float64)
    t = C.c_int32(0)
    _check(_L().orc_mpk_omp(A.n, rp, ci, va, m, X, p, Y, C.byref(t)), "mpk_omp")
    return Y, t.value


def load_bandwidth(nbytes: int = 1 << 30, reps: int = 5) -> float:
    """Host load bandwidth in bytes/s: all threads sum a buffer of nbytes, `reps` times."""
    import time
    buf = np.ones(nbytes // 8, np.float64)
    _L().orc_load_sum(buf, buf.size, 1)  # touch
    t0 = time.perf_counter()
    total = _L().orc_load_sum(buf, buf.size, reps)
    dt = time.perf_counter() - t0
    if total != float(reps) * buf.size:  # every element was read (the sum is exact below 2^53)
        raise RuntimeError(f"orc_load_sum returned {total}, expected {reps * buf.size}")
    return reps * buf.nbytes / dt


def load_sum(buf, reps: int = 1) -> float:
    """reps times the sum of a float64 buffer, over all threads (the load-bandwidth kernel)."""
    b = np.ascontiguousarray(buf, np.float64)
    return _L().orc_load_sum(b, b.size, int(reps))


def mpk_acc32(A, X, p: int) -> np.ndarray:
    """Powers with binary32 row sums over binary32-rounded inputs, binary64 vectors (the
    values of A must be exact in binary32); shape (p+1, n, m)."""
    rp, ci, va = _csr(A)
    X = _block(X, A.n)
    m = X.shape[1]
    Y = np.empty((p + 1, A.n, m), dtype=np.float64)
    _check(_L().orc_mpk_acc32(A.n, rp, ci, va, m, X, p, Y), "mpk_acc32")
    return Y


def mpk_longdouble(A, x, p: int) -> np.ndarray:
    """Single right-hand side powers accumulated in long double (error bound helper)."""
    rp, ci, va = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    Y = np.empty((p + 1, A.n), dtype=np.float64)
    _check(_L().orc_mpk_longdouble(A.n, rp, ci, va, x, p, Y), "mpk_longdouble")
    return Y


def levels(A, root: int = 0):
    """(level_of, perm, iperm, level_ptr) of the BFS levels of G(A + A^T) (Sec. 3)."""
    rp, ci, _ = _csr(A)
    n = A.n
    level_of = np.empty(n, np.int32)
    perm = np.empty(n, np.int32)
    iperm = np.empty(n, np.int32)
    level_ptr = np.empty(n + 1, np.int32)
    L = C.c_int32(0)
    _check(_L().orc_levels(n, rp, ci, root, level_of, perm, iperm, level_ptr, C.byref(L)), "levels")
    return level_of, perm, iperm, level_ptr[: L.value + 1].copy()


def permute(A, perm, iperm):
    """(row_ptr, col, val) of P A P^T with entries kept in stored order."""
    rp, ci, va = _csr(A)
    prp = np.empty(A.n + 1, np.int32)
    pci = np.empty(A.nnz, np.int32)
    pva = np.empty(A.nnz, np.float64)
    _check(_L().orc_permute(A.n, rp, ci, va, np.ascontiguousarray(perm, np.int32),
                            np.ascontiguousarray(iperm, np.int32), prp, pci, pva), "permute")
    return prp, pci, pva


def groups(level_ptr, perm_row_ptr, budget: int, val_bytes: int = 8, m: int = 1) -> np.ndarray:
    """Level indices delimiting the groups of the greedy budget rule."""
    level_ptr = np.ascontiguousarray(level_ptr, np.int32)
    L = level_ptr.size - 1
    gp = np.empty(L + 1, np.int32)
    G = C.c_int32(0)
    _check(_L().orc_groups(L, level_ptr, np.ascontiguousarray(perm_row_ptr, np.int32), val_bytes, m,
                           int(budget), gp, C.byref(G)), "groups")
    return gp[: G.value + 1].copy()


def groups_split(level_ptr, perm_row_ptr, budget: int, val_bytes: int = 8, m: int = 1) -> np.ndarray:
    """First row of every group (and n) with bulky levels cut into budget-sized pieces."""
    level_ptr = np.ascontiguousarray(level_ptr, np.int32)
    prp = np.ascontiguousarray(perm_row_ptr, np.int32)
    L = level_ptr.size - 1
    gr = np.empty(prp.size, np.int32)
    G = C.c_int32(0)
    _check(_L().orc_groups_split(L, level_ptr, prp, val_bytes, m, int(budget), gr, C.byref(G)), "groups_split")
    return gr[: G.value + 1].copy()


def lb_mpk_waves(prp, pci, pva, X, p: int, group_rows) -> np.ndarray:
    """Serial level-blocked MPK over arbitrary groups, cells in exact-dependency wave order."""
    prp = np.ascontiguousarray(prp, np.int32)
    n = prp.size - 1
    X = _block(X, n)
    m = X.shape[1]
    gr = np.ascontiguousarray(group_rows, np.int32)
    Y = np.full((p + 1, n, m), np.nan)
    _check(_L().orc_lb_mpk_waves(n, prp, np.ascontiguousarray(pci, np.int32), np.ascontiguousarray(pva, np.float64),
                                 m, X, p, gr.size - 1, gr, Y), "lb_mpk_waves")
    return Y


def lp_labels(L: int, pm: int, skew: int = 1) -> np.ndarray:
    """Execution step of each Lp-diagram cell, shape (pm, L): row p-1, column i.
    skew = 1 is the paper's diagonal order (Fig. 2); skew s walks lines i + s*p."""
    lab = np.empty(L * pm, np.int32)
    _check(_L().orc_lp_labels(L, pm, skew, lab), "lp_labels")
    return lab.reshape(pm, L)


def lb_mpk(prp, pci, pva, X, p: int, group_rows, skew: int = 1) -> np.ndarray:
    """Serial level-blocked MPK on a permuted matrix, Lp-diagram order (Sec. 3), lines g + skew*k."""
    prp = np.ascontiguousarray(prp, np.int32)
    n = prp.size - 1
    X = _block(X, n)
    m = X.shape[1]
    gr = np.ascontiguousarray(group_rows, np.int32)
    Y = np.full((p + 1, n, m), np.nan)  # a cell computed too early reads NaN
    _check(_L().orc_lb_mpk(n, prp, np.ascontiguousarray(pci, np.int32), np.ascontiguousarray(pva, np.float64),
                           m, X, p, gr.size - 1, gr, int(skew), Y), "lb_mpk")
    return Y


def cheb(A, X, degree: int, coeff_re, coeff_im=None, scale: float = 1.0, shift: float = 0.0) -> np.ndarray:
    """sum_k c_k T_k((A - shift I)/scale) X (Sec. 7 recurrence); complex when coeff_im is given."""
    rp, ci, va = _csr(A)
    X = _block(X, A.n)
    m = X.shape[1]
    cr = np.ascontiguousarray(coeff_re, np.float64)
    assert cr.size >= degree + 1
    cim = None
    if coeff_im is not None:
        cim = np.ascontiguousarray(coeff_im, np.float64)
        assert cim.size >= degree + 1
    out = np.empty((A.n, m), np.float64)
    ptr = cim.ctypes.data_as(C.c_void_p) if cim is not None else None
    _check(_L().orc_cheb(A.n, rp, ci, va, m, X, degree, cr, ptr, float(scale), float(shift), out), "cheb")
    return out


def cheb_acc32(A, X, degree: int, coeff_re, coeff_im=None, scale: float = 1.0, shift: float = 0.0) -> np.ndarray:
    """cheb() with the matrix-vector products accumulated in binary32, recurrence in binary64."""
    rp, ci, va = _csr(A)
    X = _block(X, A.n)
    m = X.shape[1]
    cr = np.ascontiguousarray(coeff_re, np.float64)
    assert cr.size >= degree + 1
    cim = None
    if coeff_im is not None:
        cim = np.ascontiguousarray(coeff_im, np.float64)
        assert cim.size >= degree + 1
    out = np.empty((A.n, m), np.float64)
    ptr = cim.ctypes.data_as(C.c_void_p) if cim is not None else None
    _check(_L().orc_cheb_acc32(A.n, rp, ci, va, m, X, degree, cr, ptr, float(scale), float(shift), out),
           "cheb_acc32")
    return out


def bessel_j(kmax: int, x: float) -> np.ndarray:
    """J_0(x)..J_kmax(x) by Miller's backward recurrence."""
    J = np.empty(kmax + 1, np.float64)
    _check(_L().orc_bessel_j(kmax, float(x), J), "bessel_j")
    return J

"""Python binding of libmpk.so, the GB300 level-blocked matrix power kernel library.

Argument marshalling only: every step of the computation runs in the CUDA library behind
the C ABI declared in include/mpk.h.  Tensors are torch CUDA tensors (torch provides
device memory and streams); calls go to the current torch stream.  If the compiled
library is missing, importing the binding's entry points raises instead of falling back.

    import paper_2405_12525_gb300 as mpk
    A = mpk.CsrMatrix(row_ptr, col, val)          # device tensors (int32, int32, float64)
    L = mpk.build_levels(A, root=0)
    P = mpk.plan(A, L, p_max=8, nrhs=1)
    Y = P.apply(X, p=8)                            # (p+1, n, nrhs), Y[k] = A^k X
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

from ._build import LIB as _LIB_PATH
from ._build import build as _build_lib

__all__ = ["build", "load", "CsrMatrix", "Levels", "Plan", "build_levels", "plan", "MpkError",
           "probe_load", "probe_dfma", "device_info", "widen_values", "BatchPlan", "batch_plan",
           "build_levels_from", "gather_rows", "spmv_rows_multi", "copy_rows",
           "EXPORTED_SYMBOLS"]

MPK_OK, MPK_ERR_INVALID, MPK_ERR_TOO_LARGE, MPK_ERR_OOM, MPK_ERR_TIMEOUT = 0, 1, 2, 3, 4
MPK_ERR_CUDA, MPK_ERR_BUDGET, MPK_ERR_UNSUPPORTED = 5, 6, 7
MPK_F64, MPK_F32, MPK_BF16 = 0, 1, 2
ORDER_ORIGINAL, ORDER_PLAN = 0, 1
ENGINE_STAGED, ENGINE_WARP, ENGINE_SWEEP = 0, 1, 2

EXPORTED_SYMBOLS = [
    "mpk_build_levels", "mpk_levels_get", "mpk_levels_destroy", "mpk_plan_opts_default", "mpk_plan",
    "mpk_plan_describe", "mpk_plan_export_csr", "mpk_plan_destroy", "mpk_apply", "mpk_spmv_powers",
    "mpk_cheb_filter", "mpk_sync_status", "mpk_probe_load", "mpk_probe_dfma", "mpk_device_info",
    "mpk_status_string", "mpk_last_error", "mpk_debug_drop_release", "mpk_read_trace", "mpk_apply_noalloc",
    "mpk_widen_values", "mpk_batch_plan", "mpk_batch_apply", "mpk_batch_describe", "mpk_batch_workspace",
    "mpk_build_levels_from", "mpk_spmv_rows", "mpk_gather_rows", "mpk_spmv_rows_multi", "mpk_copy_rows",
    "mpk_cheb_state_bytes", "mpk_cheb_begin", "mpk_cheb_advance", "mpk_cheb_finish", "mpk_apply_host",
]
MAX_ROW_SEGMENTS = 32


class MpkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mpk status {status}: {msg}")
        self.status = status


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("val_type", C.c_int32), ("is_symmetric", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("p_max", C.c_int32), ("nrhs", C.c_int32), ("cache_bytes", C.c_int64), ("order", C.c_int32),
                ("chunk_rows", C.c_int32), ("wait_limit_ns", C.c_int64), ("mem_budget", C.c_int64),
                ("trace", C.c_int32), ("level_capped", C.c_int32), ("engine", C.c_int32),
                ("shape", C.c_int32), ("shuffle_seed", C.c_int64), ("accum", C.c_int32),
                ("split_levels", C.c_int32)]


class _Desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int32), ("nrhs", C.c_int32), ("p_max", C.c_int32),
                ("order", C.c_int32), ("num_levels", C.c_int32), ("num_groups", C.c_int32),
                ("num_chunks", C.c_int32), ("group_budget_bytes", C.c_int64), ("window", C.c_int32),
                ("cache_bytes", C.c_int64),
                ("device_bytes", C.c_int64), ("padded_entries", C.c_int64),
                ("group_level_ptr_dev", C.c_void_p), ("group_row_ptr_dev", C.c_void_p),
                ("chunk_row_ptr_dev", C.c_void_p), ("perm_dev", C.c_void_p), ("shape", C.c_int32),
                ("engine", C.c_int32), ("chunk_rows", C.c_int32), ("accum", C.c_int32),
                ("split_levels", C.c_int32)]


_lib = None


def build(force: bool = False) -> str:
    """Compile libmpk.so for sm_103a (nvcc) into paper_2405_12525_gb300/_lib/."""
    return _build_lib(force=force)


def load():
    """Load libmpk.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("MPK_LIBRARY", _LIB_PATH)  # an alternative build of the same sources
    if not os.path.exists(path):
        raise RuntimeError(f"libmpk.so is missing at {path}: run paper_2405_12525_gb300.build()")
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "mpk_build_levels": [C.POINTER(_Csr), i32, vp, C.POINTER(vp)],
        "mpk_levels_get": [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                           C.POINTER(vp)],
        "mpk_plan": [C.POINTER(_Csr), vp, C.POINTER(_Opts), vp, C.POINTER(vp)],
        "mpk_plan_describe": [vp, C.POINTER(_Desc)],
        "mpk_plan_export_csr": [vp, vp, vp, vp, vp],
        "mpk_apply": [vp, vp, i32, vp, vp],
        "mpk_apply_host": [vp, vp, i32, vp, vp],
        "mpk_spmv_powers": [vp, vp, i32, vp, vp],
        "mpk_cheb_filter": [vp, vp, i32, vp, vp, dbl, dbl, vp, vp],
        "mpk_sync_status": [vp, vp],
        "mpk_probe_load": [vp, i64, i32, i32, vp, vp],
        "mpk_probe_dfma": [i32, i32, vp, vp],
        "mpk_device_info": [C.POINTER(i32), C.POINTER(i64)],
        "mpk_debug_drop_release": [vp, i32, i32],
        "mpk_read_trace": [vp, vp, vp],
        "mpk_apply_noalloc": [vp, vp, i32, vp, vp, vp],
        "mpk_widen_values": [i32, vp, i64, vp, vp],
        "mpk_batch_plan": [vp, i32, vp, C.POINTER(_Opts), vp, C.POINTER(vp)],
        "mpk_batch_apply": [vp, vp, vp, vp],
        "mpk_batch_describe": [vp, vp, vp, vp],
        "mpk_batch_workspace": [vp, C.POINTER(vp), C.POINTER(i64)],
        "mpk_build_levels_from": [vp, vp, i32, vp, C.POINTER(vp)],
        "mpk_spmv_rows": [vp, i32, i32, vp, vp, vp],
        "mpk_gather_rows": [vp, vp, i32, i32, vp, vp],
        "mpk_spmv_rows_multi": [i32, vp, vp, vp, vp, vp, vp],
        "mpk_copy_rows": [vp, vp, vp, vp, i64, i32, vp],
        "mpk_cheb_begin": [vp, vp, dbl, dbl, i32, vp, vp],
        "mpk_cheb_advance": [vp, vp, i32, i32, vp, vp, dbl, dbl, vp],
        "mpk_cheb_finish": [vp, vp, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.mpk_cheb_state_bytes.argtypes = [vp]
    lib.mpk_cheb_state_bytes.restype = C.c_int64
    lib.mpk_plan_opts_default.argtypes = [C.POINTER(_Opts)]
    lib.mpk_plan_opts_default.restype = None
    lib.mpk_levels_destroy.argtypes = [vp]
    lib.mpk_levels_destroy.restype = None
    lib.mpk_plan_destroy.argtypes = [vp]
    lib.mpk_plan_destroy.restype = None
    lib.mpk_status_string.argtypes = [C.c_int]
    lib.mpk_status_string.restype = C.c_char_p
    lib.mpk_last_error.argtypes = []
    lib.mpk_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != MPK_OK:
        lib = load()
        raise MpkError(status, (lib.mpk_last_error() or b"").decode() or lib.mpk_status_string(status).decode())


def _torch():
    import torch
    return torch


def _stream(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr()) if t is not None and t.numel() > 0 else 0


def _rows_f64(t, name: str) -> int:
    """Check a contiguous float64 CUDA tensor of rows; returns its row width (last dimension,
    1 for a vector)."""
    torch = _torch()
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return int(t.shape[-1]) if t.dim() > 1 else 1


def _index(t, dtype, name: str):
    """Check a contiguous CUDA index tensor of the given integer dtype."""
    if t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")


def _same_device(*ts):
    devs = {t.device for t in ts}
    if len(devs) > 1:
        raise ValueError(f"tensors on several devices: {sorted(str(d) for d in devs)}")


def _value_type(t) -> int:
    torch = _torch()
    types = {torch.float64: MPK_F64, torch.float32: MPK_F32, torch.bfloat16: MPK_BF16}
    if t.dtype not in types:
        raise TypeError("matrix values must be float64, float32 or bfloat16")
    return types[t.dtype]


@dataclass
class CsrMatrix:
    """Device CSR matrix: row_ptr (n+1) and col (nnz) int32 CUDA tensors, val (nnz) float64,
    float32 or bfloat16 (the plan stores values in that type and widens them exactly)."""
    row_ptr: object
    col: object
    val: object
    is_symmetric: bool = False

    @property
    def n(self) -> int:
        return int(self.row_ptr.numel()) - 1

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    def _c(self) -> _Csr:
        torch = _torch()
        vt = _value_type(self.val)
        for t, dt in ((self.row_ptr, torch.int32), (self.col, torch.int32), (self.val, self.val.dtype)):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise TypeError("CsrMatrix wants contiguous CUDA tensors: int32 row_ptr/col")
        return _Csr(self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val), vt,
                    1 if self.is_symmetric else 0)

    @staticmethod
    def from_host(A, device="cuda", is_symmetric=False, value_type=MPK_F64) -> "CsrMatrix":
        """From any object with row_ptr/col/val numpy arrays (e.g. gen.CSR); float64 values are
        rounded to nearest-even when value_type is MPK_F32 or MPK_BF16."""
        torch = _torch()
        dt = {MPK_F64: torch.float64, MPK_F32: torch.float32, MPK_BF16: torch.bfloat16}[value_type]
        return CsrMatrix(torch.as_tensor(A.row_ptr, dtype=torch.int32).to(device),
                         torch.as_tensor(A.col, dtype=torch.int32).to(device),
                         torch.as_tensor(A.val, dtype=torch.float64).to(dt).to(device), is_symmetric)


class Levels:
    """BFS levels and permutation of a matrix (owns the library handle)."""

    def __init__(self, handle, lib):
        self._h = handle
        self._lib = lib
        n, nl = C.c_int32(), C.c_int32()
        lp, pe, ip, lo = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        _check(lib.mpk_levels_get(handle, C.byref(n), C.byref(nl), C.byref(lp), C.byref(pe), C.byref(ip),
                                  C.byref(lo)))
        self.n, self.num_levels = n.value, nl.value
        self._ptrs = (lp.value, pe.value, ip.value, lo.value)

    def _view(self, ptr, count):
        return _device_i32_copy(ptr, count)

    @property
    def level_ptr(self):
        return self._view(self._ptrs[0], self.num_levels + 1)

    @property
    def perm(self):
        return self._view(self._ptrs[1], self.n)

    @property
    def iperm(self):
        return self._view(self._ptrs[2], self.n)

    @property
    def level_of(self):
        return self._view(self._ptrs[3], self.n)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.mpk_levels_destroy(self._h)
            self._h = None


class _DeviceArray:
    """Zero-copy view of library-owned device memory (CUDA array interface v3)."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _device_i32_copy(ptr: int, count: int):
    """Copy `count` int32 values of library-owned device memory into a new torch tensor."""
    torch = _torch()
    if not ptr or count == 0:
        return torch.empty(count, dtype=torch.int32, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, count, "<i4"), device="cuda").clone()


def _wrap_device_f64(ptr: int, count: int):
    """A float64 torch view (no copy) of library-owned device memory."""
    torch = _torch()
    return torch.as_tensor(_DeviceArray(ptr, count, "<f8"), device="cuda")


def build_levels_from(A: CsrMatrix, roots, stream=None) -> Levels:
    """BFS levels with the vertices `roots` (ascending) as level 0."""
    import numpy as np
    lib = load()
    r = np.ascontiguousarray(roots, dtype=np.int32)
    h = C.c_void_p()
    csr = A._c()
    _check(lib.mpk_build_levels_from(C.byref(csr), r.ctypes.data if r.size else None, int(r.size), _stream(stream),
                                     C.byref(h)))
    return Levels(h, lib)


def gather_rows(src, idx, out, stream=None):
    """out[r] = src[idx[r]] (rows of m doubles; CUDA tensors, idx int32).  The values of idx
    must be row numbers of src; they are not checked (that would need a device pass)."""
    torch = _torch()
    m = _rows_f64(src, "src")
    if _rows_f64(out, "out") != m:
        raise ValueError("src and out need rows of the same width")
    _index(idx, torch.int32, "idx")
    _same_device(src, idx, out)
    if out.numel() < idx.numel() * m:
        raise ValueError(f"out has {out.numel()} elements, the call writes {idx.numel()} rows of {m}")
    _check(load().mpk_gather_rows(_ptr(src), _ptr(idx), int(idx.numel()), m, _ptr(out), _stream(stream)))
    return out


def spmv_rows_multi(plans, row_begin, row_end, Xs, Ys, stream=None):
    """Ys[i][r] = (A_i Xs[i])[r] for plan-order rows r in [row_begin[i], row_end[i]), every
    segment in one launch (plans share value type and nrhs)."""
    n = len(plans)
    if not (len(row_begin) == len(row_end) == len(Xs) == len(Ys) == n):
        raise ValueError("one row range, X and Y per plan")
    for P, lo, hi, X, Y in zip(plans, row_begin, row_end, Xs, Ys):
        if int(hi) > int(lo):  # the library reads X and Y of non-empty segments only
            P._block(X)
            P._out_block(Y, X, 1)
    hs = (C.c_void_p * max(n, 1))(*[P._h for P in plans])
    lo = (C.c_int32 * max(n, 1))(*[int(v) for v in row_begin])
    hi = (C.c_int32 * max(n, 1))(*[int(v) for v in row_end])
    xs = (C.c_void_p * max(n, 1))(*[_ptr(X) for X in Xs])
    ys = (C.c_void_p * max(n, 1))(*[_ptr(Y) for Y in Ys])
    _check(load().mpk_spmv_rows_multi(n, hs, lo, hi, xs, ys, _stream(stream)))


def copy_rows(src, src_idx, dst, dst_idx, stream=None):
    """dst[dst_idx[t]] = src[src_idx[t]] (rows of m doubles, int64 CUDA index tensors).  The
    index values must be row numbers of src and dst, the destinations distinct; they are not
    checked (that would need a device pass)."""
    torch = _torch()
    m = _rows_f64(src, "src")
    if _rows_f64(dst, "dst") != m:
        raise ValueError("src and dst need rows of the same width")
    _index(src_idx, torch.int64, "src_idx")
    _index(dst_idx, torch.int64, "dst_idx")
    _same_device(src, src_idx, dst, dst_idx)
    if src_idx.numel() != dst_idx.numel():
        raise ValueError("one destination per source row")
    _check(load().mpk_copy_rows(_ptr(src), _ptr(src_idx), _ptr(dst), _ptr(dst_idx), int(src_idx.numel()), m,
                                _stream(stream)))
    return dst


def build_levels(A: CsrMatrix, root: int = 0, stream=None) -> Levels:
    lib = load()
    h = C.c_void_p()
    csr = A._c()
    _check(lib.mpk_build_levels(C.byref(csr), int(root), _stream(stream), C.byref(h)))
    return Levels(h, lib)


class Plan:
    """A level-blocked plan (owns the library handle)."""

    def __init__(self, handle, lib):
        self._h = handle
        self._lib = lib
        d = _Desc()
        _check(lib.mpk_plan_describe(handle, C.byref(d)))
        self.desc = d
        self.n, self.nrhs, self.p_max, self.order = d.n, d.nrhs, d.p_max, d.order

    def describe(self) -> dict:
        d = _Desc()
        _check(self._lib.mpk_plan_describe(self._h, C.byref(d)))
        return {f: getattr(d, f) for f, _ in _Desc._fields_ if not f.endswith("_dev")}

    def _device_i32(self, field: str, count: int):
        return _device_i32_copy(getattr(self.desc, field), count)

    @property
    def group_level_ptr(self):
        return self._device_i32("group_level_ptr_dev", self.desc.num_groups + 1) if self.desc.group_level_ptr_dev else None

    @property
    def group_row_ptr(self):
        return self._device_i32("group_row_ptr_dev", self.desc.num_groups + 1)

    @property
    def chunk_row_ptr(self):
        return self._device_i32("chunk_row_ptr_dev", self.desc.num_chunks + 1)

    def export_csr(self, stream=None):
        torch = _torch()
        rp = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(self.desc.nnz, dtype=torch.int32, device="cuda")
        va = torch.empty(self.desc.nnz, dtype=torch.float64, device="cuda")
        _check(self._lib.mpk_plan_export_csr(self._h, _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)))
        return rp, ci, va

    def _block(self, X):
        torch = _torch()
        if X.dtype != torch.float64 or not X.is_cuda or not X.is_contiguous():
            raise TypeError("X must be a contiguous float64 CUDA tensor")
        if X.numel() != self.n * self.nrhs:
            raise ValueError(f"X has {X.numel()} elements, plan wants n*nrhs = {self.n * self.nrhs}")

    def _out_block(self, Y, X, blocks: int, name: str = "Y"):
        """Y must hold `blocks` n x nrhs float64 blocks, contiguous, on X's device (the kernels
        write all of them)."""
        torch = _torch()
        if Y.dtype != torch.float64 or not Y.is_cuda or not Y.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
        if Y.device != X.device:
            raise ValueError(f"{name} is on {Y.device}, X on {X.device}")
        if Y.numel() < blocks * self.n * self.nrhs:
            raise ValueError(f"{name} has {Y.numel()} elements, the call writes {blocks} x n x nrhs = "
                             f"{blocks * self.n * self.nrhs}")

    def _x_clear_of_powers(self, X, Y, p: int):
        """X may be Y[0] but must not overlap Y[1..p], which the call writes while it reads X."""
        blk = 8 * self.n * self.nrhs
        x0, y1 = X.data_ptr(), Y.data_ptr() + blk
        if p > 0 and x0 < y1 + p * blk and y1 < x0 + 8 * X.numel():
            raise ValueError("X overlaps Y[1..p]")

    @staticmethod
    def _status_word(status, X):
        torch = _torch()
        if status is None:
            return None
        if status.dtype != torch.int32 or not status.is_cuda or status.numel() < 1 or status.device != X.device:
            raise TypeError("status must be an int32 CUDA tensor of at least one element on X's device")
        return _ptr(status)

    def apply(self, X, p: int, Y=None, stream=None):
        """Y[k] = A^k X, k = 0..p (level-blocked).  Returns Y of shape (p+1, n, nrhs)."""
        torch = _torch()
        self._block(X)
        if Y is None:
            Y = torch.empty((p + 1, self.n, self.nrhs), dtype=torch.float64, device=X.device)
        self._out_block(Y, X, p + 1)
        self._x_clear_of_powers(X, Y, p)
        _check(self._lib.mpk_apply(self._h, _ptr(X), int(p), _ptr(Y), _stream(stream)))
        return Y

    def apply_host(self, X, p: int, Y=None, stream=None):
        """mpk_apply with X and Y in host memory: X an n x nrhs float64 CPU tensor, Y a
        (p+1) x n x nrhs float64 pinned CPU tensor (allocated pinned if not given), in the
        plan's order.  Asynchronous on the stream: Y is complete when the stream is."""
        torch = _torch()
        if X.dtype != torch.float64 or X.is_cuda or not X.is_contiguous():
            raise TypeError("X must be a contiguous float64 CPU tensor")
        if X.numel() != self.n * self.nrhs:
            raise ValueError(f"X has {X.numel()} elements, plan wants n*nrhs = {self.n * self.nrhs}")
        if Y is None:
            Y = torch.empty((p + 1, self.n, self.nrhs), dtype=torch.float64).pin_memory()
        if Y.dtype != torch.float64 or Y.is_cuda or not Y.is_contiguous() or not Y.is_pinned():
            raise TypeError("Y must be a contiguous float64 pinned CPU tensor")
        if Y.numel() < (p + 1) * self.n * self.nrhs:
            raise ValueError(f"Y has {Y.numel()} elements, the call writes {p + 1} x n x nrhs = "
                             f"{(p + 1) * self.n * self.nrhs}")
        _check(self._lib.mpk_apply_host(self._h, _ptr(X), int(p), _ptr(Y), _stream(stream)))
        return Y

    def apply_noalloc(self, X, p: int, Y, status=None, stream=None):
        """mpk_apply without device allocation during the call (plan-order plans only).
        Y must be given; status, if given, is a one-element int32 CUDA tensor that receives
        the launch's status code."""
        self._block(X)
        self._out_block(Y, X, p + 1)
        self._x_clear_of_powers(X, Y, p)
        st = self._status_word(status, X)
        _check(self._lib.mpk_apply_noalloc(self._h, _ptr(X), int(p), _ptr(Y), st, _stream(stream)))
        return Y

    def spmv_rows(self, row_begin: int, row_end: int, X, Y, stream=None):
        """Y[r] = (A X)[r] for plan-order rows r in [row_begin, row_end) (other rows untouched)."""
        self._block(X)
        self._out_block(Y, X, 1)
        _check(self._lib.mpk_spmv_rows(self._h, int(row_begin), int(row_end), _ptr(X), _ptr(Y), _stream(stream)))
        return Y

    def spmv_powers(self, X, p: int, Y=None, stream=None):
        """Comparator: p separate SpMV launches over the same matrix copy."""
        torch = _torch()
        self._block(X)
        if Y is None:
            Y = torch.empty((p + 1, self.n, self.nrhs), dtype=torch.float64, device=X.device)
        self._out_block(Y, X, p + 1)
        self._x_clear_of_powers(X, Y, p)
        _check(self._lib.mpk_spmv_powers(self._h, _ptr(X), int(p), _ptr(Y), _stream(stream)))
        return Y

    def cheb_filter(self, X, degree: int, coeff_re, coeff_im=None, scale: float = 1.0, shift: float = 0.0,
                    out=None, stream=None):
        """sum_k c_k T_k((A - shift)/scale) X; complex coefficients act on (re, im) column pairs."""
        torch = _torch()
        import numpy as np
        self._block(X)
        cr = np.ascontiguousarray(coeff_re, dtype=np.float64)
        ci = None if coeff_im is None else np.ascontiguousarray(coeff_im, dtype=np.float64)
        if cr.size < degree + 1 or (ci is not None and ci.size < degree + 1):
            raise ValueError("need degree+1 coefficients")
        if out is None:
            out = torch.empty((self.n, self.nrhs), dtype=torch.float64, device=X.device)
        self._out_block(out, X, 1, "out")
        _check(self._lib.mpk_cheb_filter(self._h, _ptr(X), int(degree), cr.ctypes.data,
                                         ci.ctypes.data if ci is not None else None, float(scale), float(shift),
                                         _ptr(out), _stream(stream)))
        return out

    def cheb_state(self):
        """A zeroed device buffer for the resumable Chebyshev filter: (4, n, nrhs) float64."""
        torch = _torch()
        nbytes = int(self._lib.mpk_cheb_state_bytes(self._h))
        assert nbytes == 4 * self.n * self.nrhs * 8
        return torch.zeros((4, self.n, self.nrhs), dtype=torch.float64, device="cuda")

    def cheb_begin(self, X, state, c0_re: float, c0_im: float | None = None, stream=None):
        """state <- (v_0 = X, acc = c_0 X); the state then holds step 0."""
        self._block(X)
        self._out_block(state, X, 4, "state")
        _check(self._lib.mpk_cheb_begin(self._h, _ptr(X), float(c0_re), float(c0_im or 0.0),
                                        1 if c0_im is not None else 0, _ptr(state), _stream(stream)))
        return state

    def cheb_advance(self, state, k_begin: int, k_end: int, coeff_re, coeff_im=None, scale: float = 1.0,
                     shift: float = 0.0, stream=None):
        """Steps k_begin+1 .. k_end of the recurrence (absolute coefficient indices)."""
        import numpy as np
        self._out_block(state, state, 4, "state")
        cr = np.ascontiguousarray(coeff_re, dtype=np.float64)
        ci = None if coeff_im is None else np.ascontiguousarray(coeff_im, dtype=np.float64)
        if cr.size < k_end + 1 or (ci is not None and ci.size < k_end + 1):
            raise ValueError("need coefficients up to k_end")
        _check(self._lib.mpk_cheb_advance(self._h, _ptr(state), int(k_begin), int(k_end), cr.ctypes.data,
                                          ci.ctypes.data if ci is not None else None, float(scale), float(shift),
                                          _stream(stream)))
        return state

    def cheb_finish(self, state, out=None, stream=None):
        """out <- the accumulated filter (numbering as the plan's order option)."""
        torch = _torch()
        self._out_block(state, state, 4, "state")
        if out is None:
            out = torch.empty((self.n, self.nrhs), dtype=torch.float64, device=state.device)
        self._out_block(out, state, 1, "out")
        _check(self._lib.mpk_cheb_finish(self._h, _ptr(state), _ptr(out), _stream(stream)))
        return out

    def debug_drop_release(self, chunk: int, k: int):
        """Test hook: unit (chunk, k) of the next launch skips its completion flag."""
        _check(self._lib.mpk_debug_drop_release(self._h, int(chunk), int(k)))

    TRACE_FIELDS = ("units", "ctrl_poll_ns", "ctrl_poll_retries", "ctrl_slot_wait_ns", "comp_wait_ns",
                    "comp_busy_ns", "block_ns", "launches", "ctrl_stage_cyc", "ctrl_handover_cyc",
                    "ctrl_prefetch_cyc", "ctrl_decode_cyc", "comp_gather_cyc", "comp_fma_cyc",
                    "handover_lag_ns", "handover_lag_units", "block_cyc")

    def read_trace(self, stream=None) -> dict:
        """Timing counters of a plan built with trace=1 (accumulated over its launches)."""
        import numpy as np
        out = np.zeros(len(self.TRACE_FIELDS), dtype=np.int64)
        _check(self._lib.mpk_read_trace(self._h, out.ctypes.data, _stream(stream)))
        return dict(zip(self.TRACE_FIELDS, out.tolist()))

    def sync_status(self, stream=None):
        _check(self._lib.mpk_sync_status(self._h, _stream(stream)))

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.mpk_plan_destroy(self._h)
            self._h = None


def plan(A: CsrMatrix, levels: Levels | None = None, p_max: int = 8, nrhs: int = 1, cache_bytes: int = 0,
         order: int = ORDER_ORIGINAL, chunk_rows: int = 0, wait_limit_ns: int = 0, mem_budget: int = 0,
         trace: bool = False, level_capped: bool = False, engine: int = ENGINE_STAGED, shape: int = 0,
         shuffle_seed: int = 0, accum: int = MPK_F64, split_levels: bool = False, stream=None) -> Plan:
    lib = load()
    o = _Opts()
    lib.mpk_plan_opts_default(C.byref(o))
    o.p_max, o.nrhs, o.cache_bytes, o.order = p_max, nrhs, cache_bytes, order
    o.chunk_rows, o.wait_limit_ns, o.mem_budget = chunk_rows, wait_limit_ns, mem_budget
    o.trace = 1 if trace else 0
    o.level_capped = 1 if level_capped else 0
    o.engine = int(engine)
    o.shape = int(shape)
    o.shuffle_seed = int(shuffle_seed)
    o.accum = int(accum)
    o.split_levels = 1 if split_levels else 0
    h = C.c_void_p()
    csr = A._c()
    _check(lib.mpk_plan(C.byref(csr), levels._h if levels is not None else None, C.byref(o), _stream(stream),
                        C.byref(h)))
    return Plan(h, lib)


def probe_load(buf, reps: int, ctas_per_sm: int, sink, stream=None):
    """reps passes of 16-byte loads over buf (a contiguous CUDA tensor, 16-byte aligned, a
    multiple of 16 bytes); sink is an int32 CUDA tensor."""
    torch = _torch()
    if not buf.is_cuda or not buf.is_contiguous() or buf.data_ptr() % 16:
        raise TypeError("buf must be a contiguous, 16-byte aligned CUDA tensor")
    _index(sink, torch.int32, "sink")
    _check(load().mpk_probe_load(_ptr(buf), buf.numel() * buf.element_size(), reps, ctas_per_sm, _ptr(sink),
                                 _stream(stream)))


def probe_dfma(blocks: int, iters: int, sink, stream=None):
    """blocks x 256 threads of iters x 8 independent FP64 FMAs; sink is a float64 CUDA tensor."""
    _rows_f64(sink, "sink")
    _check(load().mpk_probe_dfma(blocks, iters, _ptr(sink), _stream(stream)))


class BatchPlan:
    """Plan of several matrices run together (mpk_batch_plan); owns the library handle."""

    def __init__(self, handle, lib, mats, p_each, nrhs):
        self._h = handle
        self._lib = lib
        self.sizes = [A.n for A in mats]
        self.p_each = list(p_each)
        self.nrhs = nrhs

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.mpk_plan_destroy(self._h)
            self._h = None

    def describe(self) -> dict:
        import numpy as np
        cnt = C.c_int32()
        _check(self._lib.mpk_batch_describe(self._h, C.byref(cnt), None, None))
        offs = np.zeros(cnt.value + 1, np.int32)
        pw = np.zeros(cnt.value, np.int32)
        _check(self._lib.mpk_batch_describe(self._h, None, offs.ctypes.data, pw.ctypes.data))
        d = _Desc()
        _check(self._lib.mpk_plan_describe(self._h, C.byref(d)))
        out = {f: getattr(d, f) for f, _ in _Desc._fields_ if not f.endswith("_dev")}
        out.update(count=cnt.value, row_offsets=offs.tolist(), powers=pw.tolist())
        return out

    @property
    def group_row_ptr(self):
        d = _Desc()
        _check(self._lib.mpk_plan_describe(self._h, C.byref(d)))
        return _device_i32_copy(d.group_row_ptr_dev, d.num_groups + 1)

    def views(self):
        """Block i's powers 0..p_i as a (p_i + 1, n_i, nrhs) view of the plan's workspace (plan
        order), valid until the next call on the plan (for apply(..., in_place=True))."""
        torch = _torch()
        w, stride = C.c_void_p(), C.c_int64()
        _check(self._lib.mpk_batch_workspace(self._h, C.byref(w), C.byref(stride)))
        cnt = (max(self.p_each) + 1) * stride.value
        base = _wrap_device_f64(w.value, cnt)
        out, off = [], 0
        for n, p in zip(self.sizes, self.p_each):
            out.append(torch.as_strided(base, (p + 1, n, self.nrhs), (stride.value, self.nrhs, 1), off * self.nrhs))
            off += n
        return out

    def apply(self, Xs, Ys=None, stream=None, in_place=False):
        """Ys[i] = powers 0..p_i of block i applied to Xs[i] (lists of CUDA tensors).  With
        in_place=True the powers stay in the workspace and views of it are returned."""
        torch = _torch()
        if len(Xs) != len(self.sizes):
            raise ValueError("one X per matrix")
        if in_place:
            for X, n in zip(Xs, self.sizes):
                if X.dtype != torch.float64 or not X.is_cuda or not X.is_contiguous() or X.numel() != n * self.nrhs:
                    raise TypeError("each X must be a contiguous float64 CUDA tensor of n x nrhs")
            xp = (C.c_void_p * len(Xs))(*[_ptr(X) for X in Xs])
            yp = (C.c_void_p * len(Xs))(*([None] * len(Xs)))
            _check(self._lib.mpk_batch_apply(self._h, C.cast(xp, C.c_void_p), C.cast(yp, C.c_void_p),
                                             _stream(stream)))
            return self.views()
        for X, n in zip(Xs, self.sizes):
            if X.dtype != torch.float64 or not X.is_cuda or not X.is_contiguous() or X.numel() != n * self.nrhs:
                raise TypeError("each X must be a contiguous float64 CUDA tensor of n x nrhs")
        if Ys is None:
            Ys = [torch.empty((p + 1, n, self.nrhs), dtype=torch.float64, device=X.device)
                  for X, n, p in zip(Xs, self.sizes, self.p_each)]
        if len(Ys) != len(self.sizes):
            raise ValueError("one Y per matrix")
        for X, Y, n, p in zip(Xs, Ys, self.sizes, self.p_each):
            _rows_f64(Y, "each Y")
            _same_device(X, Y)
            if Y.numel() < (p + 1) * n * self.nrhs:
                raise ValueError(f"a Y has {Y.numel()} elements, its block writes (p+1) x n x nrhs = "
                                 f"{(p + 1) * n * self.nrhs}")
        xp = (C.c_void_p * len(Xs))(*[_ptr(X) for X in Xs])
        yp = (C.c_void_p * len(Ys))(*[_ptr(Y) for Y in Ys])
        _check(self._lib.mpk_batch_apply(self._h, C.cast(xp, C.c_void_p), C.cast(yp, C.c_void_p), _stream(stream)))
        return Ys


def batch_plan(mats, p_each, p_max: int = 0, nrhs: int = 1, cache_bytes: int = 0, order: int = ORDER_ORIGINAL,
               chunk_rows: int = 0, wait_limit_ns: int = 0, mem_budget: int = 0, shape: int = 0,
               stream=None) -> BatchPlan:
    """One plan and one launch for several matrices (list of CsrMatrix, powers per matrix)."""
    lib = load()
    o = _Opts()
    lib.mpk_plan_opts_default(C.byref(o))
    o.p_max = p_max or max(p_each)
    o.nrhs, o.cache_bytes, o.order = nrhs, cache_bytes, order
    o.chunk_rows, o.wait_limit_ns, o.mem_budget = chunk_rows, wait_limit_ns, mem_budget
    o.shape = shape
    cs = (_Csr * len(mats))(*[A._c() for A in mats])
    pe = (C.c_int32 * len(mats))(*[int(p) for p in p_each])
    h = C.c_void_p()
    _check(lib.mpk_batch_plan(C.cast(cs, C.c_void_p), len(mats), C.cast(pe, C.c_void_p), C.byref(o),
                              _stream(stream), C.byref(h)))
    return BatchPlan(h, lib, mats, p_each, nrhs)


def widen_values(values, stream=None):
    """float64 copy of a float64/float32/bfloat16 CUDA tensor, widened by the library's kernels."""
    torch = _torch()
    vt = _value_type(values)
    values = values.contiguous()
    out = torch.empty(values.shape, dtype=torch.float64, device=values.device)
    _check(load().mpk_widen_values(vt, _ptr(values), values.numel(), _ptr(out), _stream(stream)))
    return out


def device_info():
    sms, l2 = C.c_int32(), C.c_int64()
    _check(load().mpk_device_info(C.byref(sms), C.byref(l2)))
    return sms.value, l2.value

"""The binding rejects tensors the library would read or write out of bounds, before any call
into the library (CPU only: a stand-in object reports a CUDA device over CPU storage, and
every case below must raise before its pointer is used)."""
import pytest
import torch

import paper_2405_12525_gb300 as mpk


class FakeCuda:
    """A CPU tensor that claims to live on cuda:0 (metadata only; never handed to the library)."""

    def __init__(self, t, device="cuda:0"):
        self._t = t
        self.dtype, self.shape = t.dtype, t.shape
        self.is_cuda = True
        self.device = torch.device(device)

    def is_contiguous(self):
        return self._t.is_contiguous()

    def dim(self):
        return self._t.dim()

    def numel(self):
        return self._t.numel()

    def data_ptr(self):
        return self._t.data_ptr()


def f64(*shape, device="cuda:0"):
    return FakeCuda(torch.zeros(shape, dtype=torch.float64), device)


def idx(n, dtype, device="cuda:0"):
    return FakeCuda(torch.zeros(n, dtype=dtype), device)


def fake_plan(n, nrhs):
    P = mpk.Plan.__new__(mpk.Plan)
    P.n, P.nrhs, P._h = n, nrhs, None
    return P


def test_gather_rows_checks():
    with pytest.raises(TypeError):  # host tensor
        mpk.gather_rows(torch.zeros(4, 2, dtype=torch.float64), idx(4, torch.int32), f64(4, 2))
    with pytest.raises(TypeError):  # 64-bit indices where the library reads 32-bit ones
        mpk.gather_rows(f64(8, 2), idx(4, torch.int64), f64(4, 2))
    with pytest.raises(ValueError):  # rows of another width
        mpk.gather_rows(f64(8, 2), idx(4, torch.int32), f64(4, 3))
    with pytest.raises(ValueError):  # out too small for the gathered rows
        mpk.gather_rows(f64(8, 2), idx(4, torch.int32), f64(3, 2))
    with pytest.raises(ValueError):  # another device
        mpk.gather_rows(f64(8, 2), idx(4, torch.int32), f64(4, 2, device="cuda:1"))


def test_copy_rows_checks():
    with pytest.raises(TypeError):  # 32-bit indices where the library reads 64-bit ones
        mpk.copy_rows(f64(8, 1), idx(4, torch.int32), f64(8, 1), idx(4, torch.int64))
    with pytest.raises(TypeError):
        mpk.copy_rows(f64(8, 1), idx(4, torch.int64), f64(8, 1), idx(4, torch.int32))
    with pytest.raises(ValueError):  # rows of another width
        mpk.copy_rows(f64(8, 2), idx(4, torch.int64), f64(8, 1), idx(4, torch.int64))
    with pytest.raises(ValueError):  # one destination per source
        mpk.copy_rows(f64(8, 1), idx(4, torch.int64), f64(8, 1), idx(3, torch.int64))
    with pytest.raises(ValueError):
        mpk.copy_rows(f64(8, 1), idx(4, torch.int64), f64(8, 1), idx(4, torch.int64, device="cuda:1"))


def test_spmv_rows_multi_checks():
    P, Q = fake_plan(10, 1), fake_plan(6, 1)
    with pytest.raises(ValueError):  # one range, X and Y per plan
        mpk.spmv_rows_multi([P, Q], [0], [1], [f64(10, 1)], [f64(10, 1)])
    with pytest.raises(ValueError):  # X of the wrong size for its plan
        mpk.spmv_rows_multi([P, Q], [0, 0], [10, 6], [f64(10, 1), f64(10, 1)], [f64(10, 1), f64(6, 1)])
    with pytest.raises(ValueError):  # Y too small
        mpk.spmv_rows_multi([P, Q], [0, 0], [10, 6], [f64(10, 1), f64(6, 1)], [f64(10, 1), f64(5, 1)])
    with pytest.raises(TypeError):  # Y not float64
        mpk.spmv_rows_multi([P], [0], [10], [f64(10, 1)], [FakeCuda(torch.zeros(10, 1))])


def test_plan_calls_check_their_outputs():
    P = fake_plan(10, 2)
    X = f64(10, 2)
    with pytest.raises(ValueError):  # Y holds p powers, the call writes p + 1
        P.apply(X, 3, Y=f64(3, 10, 2))
    with pytest.raises(ValueError):
        P.apply_noalloc(X, 3, f64(3, 10, 2))
    with pytest.raises(ValueError):
        P.spmv_powers(X, 2, Y=f64(2, 10, 2))
    with pytest.raises(ValueError):
        P.spmv_rows(0, 10, X, f64(9, 2))
    with pytest.raises(TypeError):  # status must be an int32 tensor on X's device
        P.apply_noalloc(X, 1, f64(2, 10, 2), status=torch.zeros(1, dtype=torch.int32))
    with pytest.raises(ValueError):  # X of the wrong size
        P.apply(f64(10, 1), 1, Y=f64(2, 10, 2))
    with pytest.raises(ValueError):  # Y on another device
        P.apply(X, 1, Y=f64(2, 10, 2, device="cuda:1"))
    with pytest.raises(ValueError):  # the Chebyshev state has four blocks
        P.cheb_begin(X, f64(3, 10, 2), 1.0)


def test_batch_apply_checks_its_outputs():
    B = mpk.BatchPlan.__new__(mpk.BatchPlan)
    B._h, B.sizes, B.p_each, B.nrhs = None, [5, 7], [2, 3], 1
    Xs = [f64(5, 1), f64(7, 1)]
    with pytest.raises(ValueError):  # one Y per matrix
        B.apply(Xs, [f64(3, 5, 1)])
    with pytest.raises(ValueError):  # block 1 writes 4 powers
        B.apply(Xs, [f64(3, 5, 1), f64(3, 7, 1)])
    with pytest.raises(TypeError):
        B.apply(Xs, [f64(3, 5, 1), torch.zeros(4, 7, 1, dtype=torch.float64)])
    with pytest.raises(TypeError):  # X of the wrong size
        B.apply([f64(5, 1), f64(6, 1)], [f64(3, 5, 1), f64(4, 7, 1)])


def test_probe_checks():
    with pytest.raises(TypeError):  # a 16-byte load from an unaligned address
        base = torch.zeros(64, dtype=torch.uint8)
        mpk.probe_load(FakeCuda(base[1:33]), 1, 1, idx(1, torch.int32))
    with pytest.raises(TypeError):
        mpk.probe_load(FakeCuda(torch.zeros(64, dtype=torch.uint8)), 1, 1, idx(1, torch.int64))
    with pytest.raises(TypeError):
        mpk.probe_dfma(1, 1, idx(1, torch.int32))


def test_x_may_be_y0_but_not_a_later_power():
    P = fake_plan(10, 1)
    Y = torch.zeros(4, 10, 1, dtype=torch.float64)
    with pytest.raises(ValueError, match="overlaps"):
        P.apply(FakeCuda(Y[1]), 3, Y=FakeCuda(Y))
    with pytest.raises(ValueError, match="overlaps"):
        P.spmv_powers(FakeCuda(Y[3]), 3, Y=FakeCuda(Y))
    with pytest.raises(ValueError, match="overlaps"):
        P.apply_noalloc(FakeCuda(Y.view(-1)[5:15]), 3, FakeCuda(Y))
    # X = Y[0] passes every check and reaches the library call, which the stand-in plan lacks
    with pytest.raises(AttributeError, match="_lib"):
        P.apply(FakeCuda(Y[0]), 3, Y=FakeCuda(Y))

"""Autotuner for plan parameters: the group budget C (cache_bytes), the rows per chunk, the
kernel's block shape and, for single plans, the unblocked sweep engine as one more candidate.

The paper studies p and C by hand (Sec. 6, the p x C parameter scan); here each candidate
plan is built, timed on the device with CUDA events over a few applies of the caller's
vectors, and the fastest is kept.  Works for single plans and for batch plans.
"""
from __future__ import annotations

import itertools

from . import ENGINE_SWEEP, ORDER_PLAN, batch_plan, device_info, plan


def _time(fn, reps: int):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def default_candidates():
    """Group budgets of 1/4, 1/2, 1 and 2 times the L2 size; the default chunk and 960 rows; the
    planner's block shape, shape 0 and the unstaged shape (plan option shape = 0, 1, 3)."""
    _, l2 = device_info()
    return {"cache_bytes": [l2 // 4, l2 // 2, l2, 2 * l2], "chunk_rows": [0, 960], "shape": [0, 1, 3]}


def _grid(cands):
    """Candidate options: every budget with every chunk size at the planner's shape, and with
    the default chunk size at each other shape (a shape fixes its own default chunk)."""
    for sh in cands.get("shape", [0]):
        for cb, cr in itertools.product(cands["cache_bytes"], cands["chunk_rows"] if sh == 0 else [0]):
            yield {"cache_bytes": cb, "chunk_rows": cr, "shape": sh}


def tune_plan(dA, levels, p: int, X, nrhs: int = 1, order: int = ORDER_PLAN, candidates=None, reps: int = 3):
    """Best single plan for Y = A^k X, k <= p; returns (plan, [(ms, options), ...])."""
    import torch
    cands = candidates or default_candidates()
    report, best = [], None
    Y = torch.empty((p + 1, dA.n, nrhs), dtype=torch.float64, device=X.device)
    for o in _grid(cands):
        P = plan(dA, levels, p_max=p, nrhs=nrhs, order=order, **o)
        ms = _time(lambda: P.apply(X, p, Y=Y), reps)
        P.sync_status()
        report.append((ms, o))
        if best is None or ms < best[0]:
            best = (ms, P)
        else:
            del P
    if cands.get("sweep", True):  # no level blocking: pays when the levels are too bulky
        P = plan(dA, levels, p_max=p, nrhs=nrhs, order=order, engine=ENGINE_SWEEP)
        ms = _time(lambda: P.apply(X, p, Y=Y), reps)
        P.sync_status()
        report.append((ms, {"engine": "sweep"}))
        if best is None or ms < best[0]:
            best = (ms, P)
    if best is None:
        raise ValueError("no candidate plan: the candidate lists are empty and the sweep is off")
    return best[1], sorted(report, key=lambda t: t[0])


def tune_batch(mats, p_each, Xs, nrhs: int = 1, order: int = ORDER_PLAN, candidates=None, reps: int = 3):
    """Best batch plan for the matrices; returns (batch plan, [(ms, options), ...])."""
    cands = candidates or default_candidates()
    report, best = [], None
    for o in _grid(cands):
        B = batch_plan(mats, p_each, nrhs=nrhs, order=order, **o)
        ms = _time(lambda: B.apply(Xs, in_place=True), reps)
        report.append((ms, o))
        if best is None or ms < best[0]:
            best = (ms, B)
        else:
            del B
    if best is None:
        raise ValueError("no candidate batch plan: the candidate lists are empty")
    return best[1], sorted(report, key=lambda t: t[0])

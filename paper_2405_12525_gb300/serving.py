"""Serving loop: MPK and Chebyshev-filter requests on resident matrices, continuously admitted.

Requests of different matrices, powers or degrees and widths arrive over time.  The server
keeps matrices, their BFS levels and plans on the device, admits a waiting request as soon as
a plan instance and device memory under the budget are free (a plan runs one request at a
time; a second instance is created while memory allows), runs every admitted request on its
own CUDA stream so that the work of requests in flight overlaps on the device, and records
the time from arrival to completion.  Results do not depend on what else runs: every row sum
is computed in the same order whatever the schedule.

The host logic (queue, admission, budget, completion) is separate from the device backend, so
that it can be exercised with a fake backend without a GPU.
"""
from __future__ import annotations

import heapq
import math
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    matrix: str
    kind: str                      # "mpk" (powers 0..p) or "cheb" (sum_k c_k T_k(A') X)
    order: int                     # p for "mpk", degree for "cheb"
    nrhs: int                      # right-hand sides of the request (1..8)
    x: object = None               # input block (n x nrhs), in the matrix's own numbering
    coeffs: object = None          # Chebyshev coefficients (degree + 1 reals)
    result: object = None
    t_admit: float = math.nan
    t_done: float = math.nan
    flops: float = 0.0

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


def width_bucket(nrhs: int) -> int:
    """Plans exist for 1, 2, 4 or 8 right-hand sides; a request is padded to the next one."""
    for b in (1, 2, 4, 8):
        if nrhs <= b:
            return b
    raise ValueError("at most 8 right-hand sides per request")


@dataclass(order=True)
class _Waiting:
    arrival: float
    rid: int
    req: Request = field(compare=False)


class Server:
    """Continuous admission under a device-memory budget (bytes), at most `max_inflight`
    requests in flight.  `backend` provides the device work (see GpuBackend).  keep_results:
    True keeps every result on its request, False none, a set of request ids those requests'."""

    def __init__(self, backend, hbm_budget: int, max_inflight: int = 8, keep_results=True):
        self.backend = backend
        self.keep_results = keep_results
        self.budget = int(hbm_budget)
        self.max_inflight = int(max_inflight)
        self.used = 0
        self.peak_used = 0
        self.waiting: list[_Waiting] = []
        self.inflight = []           # (request, handle, plan_key, plan, bytes)
        self.free_plans: dict = {}   # plan key -> list of idle plans
        self.plan_bytes: dict = {}   # id(plan) -> bytes
        self.done: list[Request] = []
        self.rejected: list[Request] = []  # could never fit the budget
        self.max_seen_inflight = 0

    # ------------------------------------------------------------------ plans
    def _evict(self, need: int, keep):
        """Free idle plans of other keys (largest first) until `need` more bytes fit."""
        idle = [(self.plan_bytes[id(p)], key, p) for key, ps in self.free_plans.items() if key != keep for p in ps]
        for nbytes, key, p in sorted(idle, key=lambda t: -t[0]):
            if self.used + need <= self.budget:
                break
            self.free_plans[key].remove(p)
            self.used -= nbytes
            del self.plan_bytes[id(p)]
            self.backend.drop_plan(p)

    # ------------------------------------------------------------------ requests
    def submit(self, req: Request):
        heapq.heappush(self.waiting, _Waiting(req.arrival, req.rid, req))

    def _admit(self, now: float):
        """Admit waiting requests in arrival order; one that does not fit yet does not block
        later, smaller ones.  A request needs its buffers and, unless an idle plan of its key
        exists, a new plan; idle plans of other keys are freed to make room."""
        kept = []
        while self.waiting and len(self.inflight) < self.max_inflight:
            w = heapq.heappop(self.waiting)
            req = w.req
            key = self.backend.plan_key(req)
            buf = self.backend.request_bytes(req)
            idle = self.free_plans.get(key)
            plan_need = 0 if idle else self.backend.plan_bytes(key)
            if buf + self.backend.plan_bytes(key) > self.budget:  # not even on an empty device
                req.t_done = now
                self.rejected.append(req)
                continue
            if self.used + buf + plan_need > self.budget:
                self._evict(buf + plan_need, keep=key)
            if self.used + buf + plan_need > self.budget:
                kept.append(w)
                continue
            if idle:
                plan = idle.pop()
            else:
                plan = self.backend.make_plan(key)
                nbytes = self.backend.actual_plan_bytes(plan, plan_need)
                self.plan_bytes[id(plan)] = nbytes
                self.used += nbytes
            self.used += buf
            self.peak_used = max(self.peak_used, self.used)
            req.t_admit = now
            handle = self.backend.launch(req, plan)
            self.inflight.append((req, handle, key, plan, buf))
            self.max_seen_inflight = max(self.max_seen_inflight, len(self.inflight))
        for w in kept:
            heapq.heappush(self.waiting, w)

    def _poll(self, now_fn):
        still = []
        for req, handle, key, plan, buf in self.inflight:
            if self.backend.finished(handle):
                req.t_done = now_fn()
                res = self.backend.collect(req, handle)  # also checks the request's device status
                keep = self.keep_results
                req.result = res if (keep is True or (keep and not isinstance(keep, bool) and req.rid in keep)) else None
                self.used -= buf
                self.free_plans.setdefault(key, []).append(plan)
                self.done.append(req)
            else:
                still.append((req, handle, key, plan, buf))
        self.inflight = still

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep, poll_s: float = 50e-6):
        """Replays the arrivals in real time (request.arrival seconds after the start) and
        serves until every request is done; returns the completed requests."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = clock()
        now = lambda: clock() - t0  # noqa: E731
        i = 0
        while i < len(pending) or self.waiting or self.inflight:
            t = now()
            while i < len(pending) and pending[i].arrival <= t:
                self.submit(pending[i])
                i += 1
            self._poll(now)
            self._admit(now())
            if i < len(pending) or self.waiting or self.inflight:
                sleep(poll_s)
        return self.done

    def stats(self) -> dict:
        lat = sorted(r.latency for r in self.done)
        if not lat:
            return {}
        span = max(r.t_done for r in self.done) - min(r.arrival for r in self.done)

        def pct(q):
            return lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]

        return {"requests": len(lat), "p50_ms": pct(0.50) * 1e3, "p99_ms": pct(0.99) * 1e3,
                "mean_ms": sum(lat) / len(lat) * 1e3, "max_ms": lat[-1] * 1e3,
                "throughput_rps": len(lat) / span if span > 0 else math.nan,
                "gflops": sum(r.flops for r in self.done) / span / 1e9 if span > 0 else math.nan,
                "max_inflight": self.max_seen_inflight, "peak_bytes": self.peak_used}


# Block shape of the serving plans: the unstaged shape (plan option shape=3).  Up to eight
# requests run at once, each a persistent kernel on its own stream, so the kernels share the
# SMs; blocks that stage no entries in shared memory start beside other requests' blocks.
# Config 5 at 200 requests/s served 20.9 requests/s with it against 16.8 with the staged
# shape a single launch prefers (p50 at 10 requests/s: 50 ms against 74 ms).
SERVING_SHAPE = 3


class GpuBackend:
    """Device work through the library: plans per (matrix, kind, width), one stream and one
    event per request; vectors in the matrix's own numbering."""

    def __init__(self, matrices: dict, p_max: int = 16, cheb_block: int = 8, streams: int = 8,
                 shape: int = SERVING_SHAPE):
        import torch
        from . import build_levels
        self.torch = torch
        self.mats = matrices            # name -> (CsrMatrix, scale, shift)
        self.levels = {name: build_levels(A) for name, (A, _, _) in matrices.items()}
        self.p_max = p_max
        self.cheb_block = cheb_block
        self.shape = shape              # plan option `shape` (0: the planner's choice)
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.next_stream = 0

    def plan_key(self, req):
        return (req.matrix, "mpk" if req.kind == "mpk" else "cheb", width_bucket(req.nrhs))

    def _plan_p(self, key):
        return self.p_max if key[1] == "mpk" else self.cheb_block

    def plan_bytes(self, key):
        A = self.mats[key[0]][0]
        slots = max(self._plan_p(key) + 1, 4)
        return int(12 * A.nnz * 1.05 + 8 * slots * A.n * key[2] + 64 * A.n)

    def actual_plan_bytes(self, plan, estimate):
        return int(plan.describe()["device_bytes"])

    def make_plan(self, key):
        from . import MPK_ERR_OOM, ORDER_ORIGINAL, MpkError, plan
        A = self.mats[key[0]][0]
        try:
            return plan(A, self.levels[key[0]], p_max=self._plan_p(key), nrhs=key[2], order=ORDER_ORIGINAL,
                        shape=self.shape)
        except MpkError as e:
            if e.status != MPK_ERR_OOM:
                raise
            # freed request buffers may still sit in torch's allocator cache: return them
            self.torch.cuda.synchronize()
            self.torch.cuda.empty_cache()
            return plan(A, self.levels[key[0]], p_max=self._plan_p(key), nrhs=key[2], order=ORDER_ORIGINAL,
                        shape=self.shape)

    def drop_plan(self, plan):
        del plan

    def request_bytes(self, req):
        A = self.mats[req.matrix][0]
        m = width_bucket(req.nrhs)
        out = (req.order + 1) if req.kind == "mpk" else 1
        return 8 * A.n * m * (out + 1)

    def launch(self, req, plan):
        torch = self.torch
        A, scale, shift = self.mats[req.matrix]
        m = width_bucket(req.nrhs)
        s = self.streams[self.next_stream % len(self.streams)]
        self.next_stream += 1
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            X = req.x
            if m != req.nrhs:
                X = torch.zeros((A.n, m), dtype=torch.float64, device="cuda")
                X[:, :req.nrhs] = req.x
            if req.kind == "mpk":
                Y = plan.apply(X, req.order, stream=s)
            else:
                Y = plan.cheb_filter(X, req.order, req.coeffs, scale=scale, shift=shift, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, Y, X, plan)

    def finished(self, handle):
        return handle[0].query()

    def collect(self, req, handle):
        ev, Y, X, plan = handle
        plan.sync_status()
        return Y[..., :req.nrhs] if Y.shape[-1] != req.nrhs else Y


def request_flops(A, req) -> float:
    if req.kind == "mpk":
        return 2.0 * A.nnz * req.nrhs * req.order
    return float(req.order) * req.nrhs * (2.0 * A.nnz + 6.0 * A.n)

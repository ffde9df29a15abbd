"""Host logic of the serving loop with a fake device backend and a simulated clock: admission
in arrival order under the memory budget and the in-flight limit, no head-of-line blocking,
plan reuse and eviction, rejection of requests that can never fit, latency accounting."""
import math

import pytest

from paper_2405_12525_gb300.serving import Request, Server, width_bucket


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeBackend:
    """Service time = duration per request; plan and buffer sizes from simple formulas."""

    def __init__(self, clock, plan_size=100, buf_per_order=10, duration=0.01):
        self.clock = clock
        self.plan_size = plan_size
        self.buf_per_order = buf_per_order
        self.duration = duration
        self.made, self.dropped, self.running, self.max_running = 0, 0, 0, 0

    def plan_key(self, req):
        return (req.matrix, req.kind, width_bucket(req.nrhs))

    def plan_bytes(self, key):
        return self.plan_size

    def actual_plan_bytes(self, plan, estimate):
        return estimate

    def make_plan(self, key):
        self.made += 1
        return {"key": key, "busy": False}

    def drop_plan(self, plan):
        self.dropped += 1

    def request_bytes(self, req):
        return self.buf_per_order * (req.order + 1) * width_bucket(req.nrhs)

    def launch(self, req, plan):
        assert not plan["busy"], "a plan instance runs one request at a time"
        plan["busy"] = True
        self.running += 1
        self.max_running = max(self.max_running, self.running)
        return {"end": self.clock() + self.duration * req.order, "plan": plan, "done": False}

    def finished(self, h):
        if not h["done"] and self.clock() >= h["end"]:
            h["done"] = True
            h["plan"]["busy"] = False
            self.running -= 1
        return h["done"]

    def collect(self, req, h):
        return ("result", req.rid)


def _reqs(n, gap=0.001, order=4, nrhs=2, matrices=("a", "b")):
    return [Request(i, i * gap, matrices[i % len(matrices)], "mpk" if i % 3 else "cheb", order, nrhs)
            for i in range(n)]


def test_all_served_with_latency_at_least_service_time():
    clk = Clock()
    be = FakeBackend(clk)
    srv = Server(be, hbm_budget=10_000, max_inflight=4)
    done = srv.run(_reqs(30), clock=clk, sleep=clk.sleep)
    assert len(done) == 30 and not srv.rejected
    for r in done:
        assert r.result == ("result", r.rid)
        assert r.latency >= 0.04 - 1e-9 and r.t_admit >= r.arrival
    st = srv.stats()
    assert st["requests"] == 30 and st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert srv.max_seen_inflight <= 4 and be.max_running <= 4


def test_budget_is_never_exceeded_and_limits_concurrency():
    clk = Clock()
    be = FakeBackend(clk, plan_size=100, buf_per_order=10)
    # one request: 10 * 5 * 2 = 100 bytes of buffers + a 100-byte plan per key
    srv = Server(be, hbm_budget=450, max_inflight=16)
    srv.run(_reqs(20, gap=0.0), clock=clk, sleep=clk.sleep)
    assert srv.peak_used <= 450
    assert 1 <= srv.max_seen_inflight <= 3


def test_large_request_does_not_block_small_ones():
    clk = Clock()
    be = FakeBackend(clk, plan_size=10, buf_per_order=10, duration=0.01)
    blocker = Request(0, 0.0, "c", "mpk", 20, 8)    # holds 10*21*8 = 1680 bytes for 0.2 s
    big = Request(1, 0.0005, "a", "mpk", 30, 8)     # needs 10*31*8 = 2480 bytes: waits for the blocker
    small = [Request(i, 0.001 * i, "b", "mpk", 1, 1) for i in range(2, 7)]
    srv = Server(be, hbm_budget=3000, max_inflight=8)
    done = {r.rid: r for r in srv.run([blocker, big] + small, clock=clk, sleep=clk.sleep)}
    assert len(done) == 7
    # the small requests, arriving after the big one, are served while it waits
    assert max(done[i].t_done for i in range(2, 7)) < done[1].t_admit
    assert done[1].t_admit >= done[0].t_done


def test_idle_plans_are_reused_then_evicted_for_memory():
    clk = Clock()
    be = FakeBackend(clk, plan_size=300, buf_per_order=1)
    srv = Server(be, hbm_budget=700, max_inflight=1)
    # the same key twice (reused), then a new key that only fits after evicting the idle plan
    reqs = [Request(0, 0.0, "a", "mpk", 2, 1), Request(1, 0.1, "a", "mpk", 2, 1), Request(2, 0.2, "b", "mpk", 2, 1),
            Request(3, 0.3, "c", "mpk", 2, 1)]
    srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert len(srv.done) == 4
    assert be.made == 3 and be.dropped >= 1


def test_requests_that_can_never_fit_are_rejected():
    clk = Clock()
    be = FakeBackend(clk, plan_size=100, buf_per_order=100)
    srv = Server(be, hbm_budget=500, max_inflight=4)
    reqs = [Request(0, 0.0, "a", "mpk", 10, 8), Request(1, 0.0, "a", "mpk", 1, 1)]
    srv.run(reqs, clock=clk, sleep=clk.sleep)
    assert [r.rid for r in srv.rejected] == [0] and [r.rid for r in srv.done] == [1]


def test_width_buckets():
    assert [width_bucket(k) for k in range(1, 9)] == [1, 2, 4, 4, 8, 8, 8, 8]
    with pytest.raises(ValueError):
        width_bucket(9)
    assert math.isnan(Request(0, 0.0, "a", "mpk", 1, 1).latency)


@pytest.mark.parametrize("keep,kept", [(True, set(range(12))), (False, set()), ({2, 7, 11}, {2, 7, 11})])
def test_results_kept_for_all_none_or_selected_requests(keep, kept):
    clock = Clock()
    be = FakeBackend(clock)
    srv = Server(be, hbm_budget=10 ** 6, max_inflight=4, keep_results=keep)
    done = srv.run([Request(i, 0.001 * i, "A", "mpk", 3, 1) for i in range(12)], clock=clock, sleep=clock.sleep)
    assert len(done) == 12
    assert {r.rid for r in done if r.result is not None} == kept
    assert all(r.result == ("result", r.rid) for r in done if r.result is not None)

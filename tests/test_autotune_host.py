"""Host logic of the autotuner (CPU only): the candidate grid, and the choice of the fastest
candidate with a fake planner and a fake timer in place of the device."""
import pytest
import torch

from paper_2405_12525_gb300 import autotune


def test_grid_crosses_budgets_and_chunks_at_the_planners_shape_only():
    cands = {"cache_bytes": [10, 20], "chunk_rows": [0, 960], "shape": [0, 1, 3]}
    got = list(autotune._grid(cands))
    assert got == [
        {"cache_bytes": 10, "chunk_rows": 0, "shape": 0},
        {"cache_bytes": 10, "chunk_rows": 960, "shape": 0},
        {"cache_bytes": 20, "chunk_rows": 0, "shape": 0},
        {"cache_bytes": 20, "chunk_rows": 960, "shape": 0},
        # a named shape keeps its own default chunk
        {"cache_bytes": 10, "chunk_rows": 0, "shape": 1},
        {"cache_bytes": 20, "chunk_rows": 0, "shape": 1},
        {"cache_bytes": 10, "chunk_rows": 0, "shape": 3},
        {"cache_bytes": 20, "chunk_rows": 0, "shape": 3},
    ]
    # without a shape list only the planner's choice is tried
    assert len(list(autotune._grid({"cache_bytes": [1, 2, 3], "chunk_rows": [0]}))) == 3


class FakePlan:
    def __init__(self, opts):
        self.opts = opts
        self.synced = 0

    def apply(self, X, p, Y=None):
        return Y

    def sync_status(self):
        self.synced += 1


def _fake_device(monkeypatch, ms_of):
    """plan() returns a FakePlan holding its options; _time() runs the applies and returns the
    time ms_of(options) assigns to the plan."""
    made = []

    def fake_plan(dA, levels, **kw):
        P = FakePlan(kw)
        made.append(P)
        return P

    def fake_time(fn, reps):
        assert reps >= 1
        fn()
        return ms_of(made[-1].opts)

    monkeypatch.setattr(autotune, "plan", fake_plan)
    monkeypatch.setattr(autotune, "_time", fake_time)
    return made


class Mat:
    n = 5


def test_tune_plan_keeps_the_fastest_candidate(monkeypatch):
    times = {(10, 0, 0): 3.0, (10, 960, 0): 2.5, (20, 0, 0): 1.5, (20, 960, 0): 4.0, (10, 0, 3): 2.0,
             (20, 0, 3): 1.7}

    def ms_of(o):
        if o.get("engine") == autotune.ENGINE_SWEEP:
            return 1.9
        return times[(o["cache_bytes"], o["chunk_rows"], o["shape"])]

    made = _fake_device(monkeypatch, ms_of)
    cands = {"cache_bytes": [10, 20], "chunk_rows": [0, 960], "shape": [0, 3]}
    X = torch.zeros(5, 1, dtype=torch.float64)
    best, report = autotune.tune_plan(Mat(), None, 4, X, candidates=cands)
    assert best.opts["cache_bytes"] == 20 and best.opts["chunk_rows"] == 0 and best.opts["shape"] == 0
    assert [ms for ms, _ in report] == sorted(ms for ms, _ in report)
    assert len(report) == 7 and report[0][0] == 1.5
    assert {"engine": "sweep"} in [o for _, o in report]
    assert all(P.synced == 1 for P in made)  # every candidate's status is read


def test_tune_plan_picks_the_sweep_when_it_is_fastest(monkeypatch):
    _fake_device(monkeypatch, lambda o: 0.5 if o.get("engine") == autotune.ENGINE_SWEEP else 1.0)
    X = torch.zeros(5, 1, dtype=torch.float64)
    best, report = autotune.tune_plan(Mat(), None, 4, X, candidates={"cache_bytes": [1], "chunk_rows": [0]})
    assert best.opts.get("engine") == autotune.ENGINE_SWEEP and report[0] == (0.5, {"engine": "sweep"})
    # the sweep alone still gives a plan; no candidate at all is an error, not a crash
    best, _ = autotune.tune_plan(Mat(), None, 4, X, candidates={"cache_bytes": [], "chunk_rows": [0]})
    assert best.opts.get("engine") == autotune.ENGINE_SWEEP
    with pytest.raises(ValueError):
        autotune.tune_plan(Mat(), None, 4, X, candidates={"cache_bytes": [], "chunk_rows": [0], "sweep": False})


def test_tune_batch_keeps_the_fastest_candidate(monkeypatch):
    made = []

    class FakeBatch:
        def __init__(self, kw):
            self.opts = kw

        def apply(self, Xs, in_place=False):
            assert in_place
            return Xs

    def fake_batch_plan(mats, p_each, **kw):
        made.append(FakeBatch(kw))
        return made[-1]

    monkeypatch.setattr(autotune, "batch_plan", fake_batch_plan)
    monkeypatch.setattr(autotune, "_time", lambda fn, reps: (fn(), 10.0 / made[-1].opts["cache_bytes"])[1])
    best, report = autotune.tune_batch([Mat()], [3], [None], candidates={"cache_bytes": [1, 4, 2], "chunk_rows": [0]})
    assert best.opts["cache_bytes"] == 4 and [ms for ms, _ in report] == [2.5, 5.0, 10.0]
    with pytest.raises(ValueError):
        autotune.tune_batch([Mat()], [3], [None], candidates={"cache_bytes": [], "chunk_rows": [0]})

"""Host logic of the serving loop (admission, HBM budget, LRU eviction, per-state
ordering) on the CPU: the solver contexts and CUDA streams are replaced by fakes
that record when each request runs, so no GPU and no library are needed."""
import contextlib
import threading
import time

import pytest

torch = pytest.importorskip("torch")

from paper_2505_24504_gb300 import jfnk, serve  # noqa: E402


class _FakeStats:
    status = 0
    gmres_its = 3


class _FakeContext:
    live = 0
    peak = 0
    lock = threading.Lock()
    log = []

    def __init__(self, grid, k, phys, opts):
        self.sid = grid
        with _FakeContext.lock:
            _FakeContext.live += 1
            _FakeContext.peak = max(_FakeContext.peak, _FakeContext.live)

    @staticmethod
    def workspace_bytes(grid, k, opts=None):
        return 100 * k

    def implicit_step(self, U, dt, scheme=1, raise_on_error=True):
        t0 = time.perf_counter()
        time.sleep(0.002)
        with _FakeContext.lock:
            _FakeContext.log.append((self.sid, U["n"], t0, time.perf_counter()))
        U["n"] += 1
        return _FakeStats()

    def close(self):
        with _FakeContext.lock:
            _FakeContext.live -= 1


class _FakeStream:
    def synchronize(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    monkeypatch.setattr(jfnk, "Context", _FakeContext)
    monkeypatch.setattr(torch.cuda, "Stream", _FakeStream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    _FakeContext.live = _FakeContext.peak = 0
    _FakeContext.log = []
    yield


def _states(n):
    # state sid: "grid" = sid (the fake context remembers it), order k = 1 + sid % 3,
    # footprint 100 k bytes; U counts the steps applied to it
    return {sid: serve.StateSpec(grid=sid, k=1 + sid % 3, phys=None, opts=None, dt=1.0, scheme=1,
                                 U={"n": 0})
            for sid in range(n)}


def test_budget_eviction_and_per_state_order(fakes):
    states = _states(8)
    budget = 450                      # room for about two of the eight contexts at once
    arrivals = [(0.001 * i, i % 8) for i in range(64)]
    srv = serve.Server(states, hbm_budget=budget, workers=4)
    rep = srv.run(arrivals, timeout_s=60.0)
    srv.close()
    s = rep.summary()
    assert s["requests"] == 64 and s["failed"] == 0
    assert rep.peak_bytes <= budget
    assert rep.contexts_evicted > 0 and rep.contexts_created > 8
    assert _FakeContext.live == 0
    # every request of a state ran, one at a time, in arrival order
    for sid, st in states.items():
        runs = sorted((t0, t1, n) for (i, n, t0, t1) in _FakeContext.log if i == sid)
        assert [n for (_, _, n) in runs] == list(range(8))
        assert all(runs[q][1] <= runs[q + 1][0] for q in range(len(runs) - 1))
        assert st.steps_done == 8 and st.U["n"] == 8
    for r in rep.records:
        assert r.end >= r.start >= r.arrival


def test_contexts_kept_when_budget_allows(fakes):
    states = _states(4)
    arrivals = [(0.0005 * i, i % 4) for i in range(40)]
    srv = serve.Server(states, hbm_budget=10_000, workers=3)
    rep = srv.run(arrivals, timeout_s=60.0)
    srv.close()
    assert rep.summary()["failed"] == 0
    assert rep.contexts_created == 4 and rep.contexts_evicted == 0
    assert rep.max_concurrent <= 3


def test_state_larger_than_budget_is_rejected(fakes):
    with pytest.raises(ValueError):
        serve.Server(_states(3), hbm_budget=250, workers=2)   # state 2 needs 300 bytes


def test_failed_step_is_retried_with_substeps(fakes, monkeypatch):
    # a step longer than 0.3 fails with ENAN (state untouched, as the library
    # restores U^n): the server retries the request as 2, then 4 substeps
    class _Stats:
        def __init__(self, status):
            self.status = status
            self.gmres_its = 1

    def step(self, U, dt, scheme=1, raise_on_error=True):
        # state 3 fails on its second substep at dt/2: the partial progress must be undone
        if dt > 0.3 or (U.get("flaky") and U["n"] == 1 and dt > 0.3 / 2):
            return _Stats(-6)
        U["n"] += 1
        return _Stats(0)

    monkeypatch.setattr(_FakeContext, "implicit_step", step)
    states = {0: serve.StateSpec(grid=0, k=1, phys=None, opts=None, dt=1.0, scheme=1, U={"n": 0}),
              1: serve.StateSpec(grid=1, k=1, phys=None, opts=None, dt=0.25, scheme=1, U={"n": 0}),
              2: serve.StateSpec(grid=2, k=1, phys=None, opts=None, dt=8.0, scheme=1, U={"n": 0}),
              3: serve.StateSpec(grid=3, k=1, phys=None, opts=None, dt=0.5, scheme=1, U={"n": 0, "flaky": 1})}
    srv = serve.Server(states, hbm_budget=10_000, workers=2)
    rep = srv.run([(0.0, 0), (0.0, 1), (0.0, 2), (0.0, 3)], timeout_s=30.0)
    srv.close()
    by = {r.sid: r for r in rep.records}
    assert by[0].status == 0 and by[0].substeps == 4 and states[0].U["n"] == 4
    assert by[1].status == 0 and by[1].substeps == 1 and states[1].U["n"] == 1
    assert by[2].status == -6 and states[2].U["n"] == 0          # dt/4 = 2 still too long: reported
    s = rep.summary()
    # state 3: dt = 0.5 fails, 2 x 0.25 fails at the second substep (undone), 4 x 0.125 succeeds
    assert by[3].status == 0 and by[3].substeps == 4 and states[3].U["n"] == 4
    assert s["failed"] == 1 and s["failed_by_state"] == {2: {-6: 1}} and s["retried_with_substeps"] == 3

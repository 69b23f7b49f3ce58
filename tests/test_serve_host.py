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

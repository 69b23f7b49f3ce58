"""Request loop for implicit-step requests on device-resident atmospheric states
(continuous batching, not a queue alone).

* States stay on the device between requests (one FP64 DG vector each).
* A request asks for one implicit step of one state.  It is admitted when a
  worker slot is free, no earlier request of the same state is in flight, and
  the HBM budget has room for that state's solver context (Krylov basis, FV
  levels, workspace: `Context.workspace_bytes`).  Contexts are created on
  admission and kept while idle; idle contexts are destroyed least-recently-used
  first when a new context needs room.
* Admitted requests run concurrently: each worker thread drives the C-ABI
  implicit step on its own CUDA stream (the binding releases the GIL), so
  requests that arrive while others are on the GPU overlap on the device.
* A state's requests run in arrival order and one at a time, and every
  kernel is deterministic, so each result is bit-identical to stepping that
  state alone.
* A step that does not converge (the library restores U^n) is retried over the
  same interval as 2, then 4 substeps; the report counts such requests.

Latency = completion - arrival (wall clock); the report gives p50 / p99 and the
sustained steps/s.  Scheduling is host logic; every solve runs in libjfnk.so.
"""
from __future__ import annotations

import collections
import copy
import threading
import time
from dataclasses import dataclass, field

from . import jfnk


def _copy_state(U):
    return U.clone() if hasattr(U, "clone") else copy.deepcopy(U)


def _restore_state(U, snap):
    if hasattr(U, "copy_"):
        U.copy_(snap)
    else:
        U.clear()
        U.update(copy.deepcopy(snap))


@dataclass
class StateSpec:
    """A resident state: solver construction arguments plus its device vector."""
    grid: "jfnk.Grid"
    k: int
    phys: "jfnk.Physics"
    opts: "jfnk.Opts"
    dt: float
    scheme: int
    U: object            # torch CUDA float64 tensor, the state U' (updated in place)
    steps_done: int = 0

    @property
    def footprint(self) -> int:
        return jfnk.Context.workspace_bytes(self.grid, self.k, self.opts)


@dataclass
class Record:
    sid: int
    arrival: float
    start: float = 0.0
    end: float = 0.0
    status: int = 0
    gmres_its: int = 0
    substeps: int = 1


@dataclass
class Report:
    records: list
    wall_s: float
    peak_bytes: int
    contexts_created: int
    contexts_evicted: int
    max_concurrent: int
    extra: dict = field(default_factory=dict)

    def latencies(self):
        return sorted(r.end - r.arrival for r in self.records)

    def percentile(self, p):
        lat = self.latencies()
        if not lat:
            return 0.0
        i = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
        return lat[i]

    def summary(self):
        n = len(self.records)
        return {"requests": n, "steps_per_s": n / self.wall_s if self.wall_s > 0 else 0.0,
                "p50_ms": 1e3 * self.percentile(50), "p99_ms": 1e3 * self.percentile(99),
                "wall_s": self.wall_s, "peak_context_bytes": self.peak_bytes,
                "contexts_created": self.contexts_created, "contexts_evicted": self.contexts_evicted,
                "max_concurrent": self.max_concurrent,
                "failed": sum(1 for r in self.records if r.status != 0),
                "failed_by_state": self.failures(),
                "retried_with_substeps": sum(1 for r in self.records if r.substeps > 1)}

    def failures(self):
        """{state id: {status code: requests}} of the requests that did not succeed."""
        out = {}
        for r in self.records:
            if r.status != 0:
                d = out.setdefault(r.sid, {})
                d[r.status] = d.get(r.status, 0) + 1
        return out


class Server:
    def __init__(self, states: dict, hbm_budget: int, workers: int = 8):
        self.states = states
        self.budget = int(hbm_budget)
        self.workers = int(workers)
        self._ctx = collections.OrderedDict()   # sid -> Context (LRU order)
        self._busy = set()
        self._lock = threading.Condition()
        self._bytes = 0
        self.peak = 0
        self.created = 0
        self.evicted = 0
        for sid, st in states.items():
            if st.footprint > self.budget:
                raise ValueError(f"state {sid} needs {st.footprint} bytes, budget is {self.budget}")

    # -- admission (called with the lock held) -------------------------------
    def _can_admit(self, sid) -> bool:
        if sid in self._busy:
            return False
        if sid in self._ctx:
            return True
        need = self.states[sid].footprint
        free = self.budget - self._bytes
        if need <= free:
            return True
        idle = [s for s in self._ctx if s not in self._busy]
        return need <= free + sum(self.states[s].footprint for s in idle)

    def _acquire(self, sid):
        if sid in self._ctx:
            self._ctx.move_to_end(sid)
            ctx = self._ctx[sid]
        else:
            need = self.states[sid].footprint
            for s in list(self._ctx):
                if self._bytes + need <= self.budget:
                    break
                if s in self._busy:
                    continue
                self._ctx.pop(s).close()
                self._bytes -= self.states[s].footprint
                self.evicted += 1
            st = self.states[sid]
            ctx = jfnk.Context(st.grid, st.k, st.phys, st.opts)
            self._ctx[sid] = ctx
            self._bytes += need
            self.created += 1
            self.peak = max(self.peak, self._bytes)
        self._busy.add(sid)
        return ctx

    # Step-size fallback: when a step fails to converge (Newton or GMRES cap, a
    # non-finite norm) the library has restored U^n, and the request is retried as
    # 2, then 4 substeps of dt/2, dt/4 (the same time interval); the record keeps
    # the number of substeps it took.
    RETRY_CODES = (-4, -6)          # JFNK_ENOTCONV, JFNK_ENAN
    MAX_HALVINGS = 2

    def _step(self, ctx, st, stream):
        """One request: returns (status, GMRES iterations, substeps).  A failed
        substep sequence is undone from a copy of U^n before the next try."""
        snap = None
        for h in range(self.MAX_HALVINGS + 1):
            n = 1 << h
            if h == 1:
                snap = _copy_state(st.U)
            elif h > 1:
                _restore_state(st.U, snap)
            its, status = 0, 0
            for _ in range(n):
                s = ctx.implicit_step(st.U, st.dt / n, scheme=st.scheme, raise_on_error=False)
                stream.synchronize()
                its += s.gmres_its
                status = s.status
                if status != 0:
                    break
            if status == 0 or status not in self.RETRY_CODES:
                return status, its, n
        if snap is not None:
            _restore_state(st.U, snap)
        return status, its, n

    def run(self, arrivals, timeout_s: float = 600.0):
        """Replay (arrival_time_s, sid) requests in real time; returns a Report.
        Raises RuntimeError if the workers do not finish within timeout_s."""
        import torch
        reqs = sorted(arrivals)
        pending = collections.deque()
        records = []
        t0 = time.perf_counter()
        state = {"next": 0, "done": 0, "inflight": 0, "maxc": 0}
        total = len(reqs)

        def pick():
            # first pending request whose state can be admitted (FIFO per state)
            seen = set()
            for i, rec in enumerate(pending):
                if rec.sid in seen:
                    continue
                seen.add(rec.sid)
                if self._can_admit(rec.sid):
                    del pending[i]
                    return rec
            return None

        def worker():
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                while True:
                    with self._lock:
                        while True:
                            now = time.perf_counter() - t0
                            while state["next"] < total and reqs[state["next"]][0] <= now:
                                a, sid = reqs[state["next"]]
                                pending.append(Record(sid=sid, arrival=a))
                                state["next"] += 1
                            if state["done"] == total:
                                self._lock.notify_all()
                                return
                            rec = pick()
                            if rec is not None:
                                try:
                                    ctx = self._acquire(rec.sid)
                                except Exception as exc:   # admission failed: record, never hang
                                    rec.status = getattr(exc, "code", -3)
                                    rec.start = rec.end = time.perf_counter() - t0
                                    state["done"] += 1
                                    records.append(rec)
                                    self._lock.notify_all()
                                    continue
                                state["inflight"] += 1
                                state["maxc"] = max(state["maxc"], state["inflight"])
                                break
                            wait = None
                            if state["next"] < total:
                                wait = max(0.0, reqs[state["next"]][0] - now)
                            self._lock.wait(timeout=wait if wait is not None else 0.05)
                    st = self.states[rec.sid]
                    rec.start = time.perf_counter() - t0
                    try:
                        rec.status, rec.gmres_its, rec.substeps = self._step(ctx, st, stream)
                    except Exception as exc:   # a failed request must not stop the loop
                        rec.status = getattr(exc, "code", -3)
                    rec.end = time.perf_counter() - t0
                    with self._lock:
                        st.steps_done += 1
                        self._busy.discard(rec.sid)
                        state["inflight"] -= 1
                        state["done"] += 1
                        records.append(rec)
                        self._lock.notify_all()

        threads = [threading.Thread(target=worker, daemon=True) for _ in range(self.workers)]
        for t in threads:
            t.start()
        deadline = time.perf_counter() + timeout_s
        for t in threads:
            t.join(timeout=max(0.0, deadline - time.perf_counter()))
        if any(t.is_alive() for t in threads):
            raise RuntimeError(f"serving loop did not finish within {timeout_s} s "
                               f"({state['done']} of {total} requests done)")
        wall = time.perf_counter() - t0
        return Report(records=records, wall_s=wall, peak_bytes=self.peak, contexts_created=self.created,
                      contexts_evicted=self.evicted, max_concurrent=state["maxc"])

    def close(self):
        with self._lock:
            for c in self._ctx.values():
                c.close()
            self._ctx.clear()
            self._bytes = 0


# ---- member-sharded serving over several GPUs ---------------------------------
# States are independent, so N GPUs serve N disjoint partitions of them: rank r
# owns every state id with sid % world == r and serves only the requests for
# those states, each rank with its own Server on its own device.  Nothing is
# exchanged on the data path; the ranks meet once at the end to pool their
# latency records for the report.

def shard_states(states: dict, rank: int, world: int) -> dict:
    """The states rank `rank` of `world` owns (sid % world == rank)."""
    return {sid: st for sid, st in states.items() if sid % world == rank}


def shard_requests(arrivals, rank: int, world: int):
    """The requests for the states rank `rank` owns, arrival times unchanged."""
    return [(t, sid) for (t, sid) in arrivals if sid % world == rank]


def pooled_summary(report: "Report", dist=None) -> dict:
    """Whole-job summary over all ranks: every rank's latencies pooled (one
    all_gather_object at the end, outside the data path), steps/s = all requests
    over the longest rank's wall time.  With dist None: this rank alone."""
    lat = [r.end - r.arrival for r in report.records]
    failed = sum(1 for r in report.records if r.status != 0)
    parts = [(lat, report.wall_s, failed)]
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, (lat, report.wall_s, failed))
    allat = sorted(x for p in parts for x in p[0])
    wall = max(p[1] for p in parts)

    def pct(q):
        if not allat:
            return 0.0
        return allat[min(len(allat) - 1, max(0, int(round(q / 100.0 * (len(allat) - 1)))))]

    return {"requests": len(allat), "steps_per_s": len(allat) / wall if wall > 0 else 0.0,
            "p50_ms": 1e3 * pct(50), "p99_ms": 1e3 * pct(99), "wall_s": wall,
            "failed": sum(p[2] for p in parts), "ranks": len(parts)}

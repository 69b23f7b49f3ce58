"""Member-sharded serving on world_size 2 (gloo, CPU): each rank serves only the
states it owns, every request is served exactly once across the ranks, nothing
is exchanged while serving, and the pooled p50/p99 equal the percentiles of
the union of both ranks' latencies.  The solver contexts are fakes, so this
covers the host logic only (multi-GPU serving is unmeasured on hardware)."""
import os
import socket
import time

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import contextlib
    import threading

    from paper_2505_24504_gb300 import jfnk, serve

    class FakeStats:
        status = 0
        gmres_its = 1

    class FakeContext:
        def __init__(self, grid, k, phys, opts):
            self.sid = grid

        @staticmethod
        def workspace_bytes(grid, k, opts=None):
            return 100

        def implicit_step(self, U, dt, scheme=1, raise_on_error=True):
            time.sleep(0.001 * (1 + self.sid % 3))
            U["n"] += 1
            U["rank"].add(rank)
            return FakeStats()

        def close(self):
            pass

    class FakeStream:
        def synchronize(self):
            pass

    jfnk.Context = FakeContext
    torch.cuda.Stream = FakeStream
    torch.cuda.stream = lambda s: contextlib.nullcontext()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    states = {sid: serve.StateSpec(grid=sid, k=1, phys=None, opts=None, dt=1.0, scheme=1,
                                   U={"n": 0, "rank": set()}) for sid in range(7)}
    arrivals = [(0.0007 * i, (3 * i) % 7) for i in range(60)]
    mine = serve.shard_states(states, rank, world)
    reqs = serve.shard_requests(arrivals, rank, world)
    srv = serve.Server(mine, hbm_budget=10_000, workers=3)
    rep = srv.run(reqs, timeout_s=60.0)
    srv.close()
    pooled = serve.pooled_summary(rep, dist)
    lat = [r.end - r.arrival for r in rep.records]
    out[rank] = {"owned": sorted(mine), "served": sorted(r.sid for r in rep.records),
                 "steps": {sid: st.U["n"] for sid, st in mine.items()},
                 "ranks_touching": {sid: sorted(st.U["rank"]) for sid, st in mine.items()},
                 "lat": lat, "pooled": pooled, "n_req": len(reqs)}
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_serving_gloo():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    r0, r1 = out[0], out[1]
    assert r0["owned"] == [0, 2, 4, 6] and r1["owned"] == [1, 3, 5]
    assert set(r0["served"]) <= set(r0["owned"]) and set(r1["served"]) <= set(r1["owned"])
    assert r0["n_req"] + r1["n_req"] == 60
    assert len(r0["served"]) + len(r1["served"]) == 60
    for r, rank in ((r0, 0), (r1, 1)):
        for sid, touched in r["ranks_touching"].items():
            assert touched in ([], [rank])          # a state is stepped by its owner only
        assert sum(r["steps"].values()) == r["n_req"]
    allat = sorted(r0["lat"] + r1["lat"])
    want50 = allat[int(round(0.5 * (len(allat) - 1)))]
    want99 = allat[int(round(0.99 * (len(allat) - 1)))]
    for r in (r0, r1):
        p = r["pooled"]
        assert p["requests"] == 60 and p["ranks"] == 2 and p["failed"] == 0
        assert abs(p["p50_ms"] - 1e3 * want50) < 1e-9 and abs(p["p99_ms"] - 1e3 * want99) < 1e-9

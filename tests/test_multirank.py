"""The N > 1 path of bench.py (one replica per rank, barrier-bracketed timing,
max over ranks, whole-job aggregate) with world_size 2 on the gloo backend, CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    my_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(my_ms, dist, device="cpu")
    rate = bench.whole_job_rate(10, ms, world)
    out[rank] = (ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, rate = out[0]
    assert ms == 150.0
    assert abs(rate - 2 * 10 / 0.150) < 1e-9

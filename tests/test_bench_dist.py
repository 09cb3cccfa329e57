"""The benchmark's multi-rank aggregation on CPU: two gloo ranks, each reporting its own
decodes and time; the whole-job value is all decodes over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dec, sec = bench.aggregate(dist, 1000.0 * (rank + 1), 2.0 + rank, device="cpu")
    out[rank] = (dec, sec)
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (3000.0, 3.0)


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(None, 5.0, 2.0) == (5.0, 2.0)

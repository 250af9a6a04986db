"""The multi-GPU path of the benchmark and of the serving loop is replicas only
(independent problems share nothing): two gloo ranks on the CPU check the
max-over-ranks timing aggregation and the request sharding."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r "took" 1 + r seconds for 100 * (r + 1) units
        t, rate = bench.aggregate(1.0 + rank, 100.0 * (rank + 1), dist)
        # requests split across replicas, every one served exactly once
        mine = bench.shard(list(range(11)), rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = (t, rate, sorted(sum(gathered, [])))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_and_sharding():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, rate, served = res[rank]
        assert t == 2.0                      # the slowest rank
        assert rate == pytest.approx(300.0 / 2.0)  # all units over that time
        assert served == list(range(11))

"""The multi-replica path of the benchmark (one process per GPU, weak
scaling, time = max over ranks) exercised on CPU with gloo, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 100.0 + 50.0 * rank              # rank 1 is the slow one
    total, value = bench.aggregate(local, count_per_rank=4096, steps=5, world=world, dist=dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, total, value, bench.dist_info()))


def test_two_replicas_aggregate_with_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, total, value, info in res:
        assert total == 150.0                 # the slowest rank
        assert abs(value - 4096 * 2 * 5 / 0.150) < 1e-6
        assert info == (rank, 2, rank)

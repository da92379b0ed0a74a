"""Multi-rank path of the benchmark (replicas: one process per GPU, no data
exchange): the throughput reduction over ranks, run as world-size-2 gloo
ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed (r + 1) * 1000 points in (r + 1) * 0.5 s
        value, tmax = bench.replica_throughput((rank + 1) * 1000, (rank + 1) * 0.5)
        q.put((rank, value, tmax))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_world2_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for _, value, tmax in out:
        assert tmax == pytest.approx(1.0)
        assert value == pytest.approx(3000 / 1.0)


def test_replica_throughput_single_process():
    import bench
    v, t = bench.replica_throughput(500, 0.25)
    assert v == pytest.approx(2000.0) and t == 0.25

"""The multi-GPU path of the benchmark is replicas only: each rank solves its own problem and the
ranks meet only in a barrier and a max-reduction of the elapsed time. Its host logic runs here on
CPU with two gloo ranks."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    units = 1000.0
    elapsed = 2.0 + rank  # rank 1 is the slowest: 3 s
    value = bench.replica_throughput(units, elapsed)
    slowest = bench.max_over_ranks(elapsed)
    dist.barrier()
    out.put((rank, value, slowest))
    dist.destroy_process_group()


def test_two_rank_replica_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest in res:
        assert slowest == pytest.approx(3.0)
        assert value == pytest.approx(2 * 1000.0 / 3.0)  # all ranks' units over the slowest time


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.replica_throughput(100.0, 2.0) == pytest.approx(50.0)

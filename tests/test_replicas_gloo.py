"""Multi-GPU runs are independent replicas (no collective on the data path):
the bench takes the slowest rank's time and counts one evaluation per rank.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [1500.0, 2500.0][rank]
    ms = bench.reduce_max(local_ms, world)
    q.put((rank, ms, bench.replica_throughput(ms, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, thr in out:
        assert ms == 2500.0
        assert thr == pytest.approx(2 / 2.5)


def test_single_process_is_unchanged():
    import bench

    assert bench.reduce_max(123.0, 1) == 123.0
    assert bench.replica_throughput(500.0, 1) == pytest.approx(2.0)

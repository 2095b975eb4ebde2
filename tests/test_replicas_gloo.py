"""The N > 1 path of bench.py runs independent replicas: the whole-job
throughput is N x the work of one replica over the slowest replica's time.
Checked with two gloo ranks on the CPU (127.0.0.1 rendezvous)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, t = bench.aggregate(times[rank], 2.0e9, 10, dist, "cpu")
    out[rank] = (value, t)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    times = [1.0, 2.0]                      # rank 1 is slower
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        value, t = out[r]
        assert t == 2.0
        assert value == pytest.approx(2 * 2.0e9 * 10 / 2.0 / 1e9)


def test_single_replica_needs_no_process_group():
    import bench
    value, t = bench.aggregate(0.5, 1.0e9, 4)
    assert t == 0.5 and value == pytest.approx(8.0)

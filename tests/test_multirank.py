"""The N > 1 path of bench.py (independent replicas, one per rank) on CPU:
two gloo ranks agree on the slowest rank's time and on the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.5 + rank, torch.device("cpu"))
    v = bench.replica_throughput(1024 * 10, world, t)
    dist.barrier()
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, v = res[rank]
        assert t == pytest.approx(2.5)
        assert v == pytest.approx(2 * 1024 * 10 / 2.5)


def test_single_process_passthrough():
    import torch
    import bench
    assert bench.max_over_ranks(3.25, torch.device("cpu")) == 3.25
    assert bench.replica_throughput(100, 1, 2.0) == 50.0

"""N > 1: the benchmark runs independent replicas (one GPU per replica, no
data exchange between them); the whole-job value is the units of all ranks
over the slowest rank's time.  Two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 5.0][rank]
    units = [100.0, 300.0][rank]
    value, tmax, total = bench.aggregate_replicas(seconds, units, torch.device("cpu"))
    q.put((rank, value, tmax, total))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, tmax, total in res:
        assert tmax == 5.0 and total == 400.0
        assert value == pytest.approx(80.0)


def test_single_process_aggregation():
    import bench
    assert bench.aggregate_replicas(2.0, 10.0) == (5.0, 2.0, 10.0)

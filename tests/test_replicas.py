"""The multi-GPU path is replicas only (independent instances, no value
crosses GPUs): bench.py's whole-job aggregation over ranks, run as two gloo
processes on the CPU."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took r+1 seconds for 1000 units: the job rate uses the slowest rank
    rate = bench.replica_rate(dist, world, 1000, float(rank + 1))
    slowest = bench.max_over_ranks(dist, float(rank + 1))
    bench.barrier(dist)
    out[rank] = (rate, slowest)
    dist.destroy_process_group()


def test_replica_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (2 * 1000 / 2.0, 2.0)


def test_replica_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_rate(None, 1, 500, 2.0) == 250.0

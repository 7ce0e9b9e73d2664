"""The N>1 path of bench.py: independent replicas, throughput = units of all ranks / max time,
checked with two gloo ranks on the CPU (no GPU, no NCCL)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [400.0, 500.0][rank]             # rank 1 is slower
    value, ms_max = bench.aggregate(ms, 8, dist)
    q.put((rank, value, ms_max))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    for rank, value, ms_max in res:
        assert ms_max == 500.0
        assert value == pytest.approx(16 / 0.5)       # 2 ranks x 8 units in the slowest time


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(250.0, 8) == (32.0, 250.0)

"""The multi-GPU path of bench.py is independent replicas: the only
collective is the MAX over ranks of the timed region. Checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 1000.0 * (rank + 1)            # rank 1 is the slowest: 2000 ms
    value, total = bench.aggregate_replicas(local_ms, steps=10, world=world, device=torch.device("cpu"))
    out[rank] = (value, total)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            value, total = out[r]
            assert total == pytest.approx(2000.0)
            assert value == pytest.approx(10 * 2 / 2.0)   # 20 solves in 2 s


def test_single_rank_needs_no_collective():
    import bench
    value, total = bench.aggregate_replicas(500.0, steps=5, world=1, device=torch.device("cpu"))
    assert total == 500.0 and value == pytest.approx(10.0)

"""bench.py's N > 1 path on CPU: two gloo ranks run independent replicas;
the whole-job value is the sum of the ranks' units over the slowest rank's
time, identical on every rank."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [1000.0, 1250.0][rank]
    value, ms = bench.aggregate(local_ms, 8.0, world, device="cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        value, ms = out[r]
        assert ms == 1250.0                      # the slowest rank
        assert value == pytest.approx(16.0 / 1.25)  # all ranks' units / max time


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(500.0, 4.0, 1) == (8.0, 500.0)

"""The N > 1 path of bench.py on CPU: world_size 2 over gloo (replicas only --
no data-path collective; the only collective is the max of the per-rank step
time, and the whole-job value counts every rank's solves)."""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, ms, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.max_over_ranks(ms[rank], dist, torch.device("cpu"))
    q.put((rank, m, bench.replica_value(world, m)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_replica_value(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ms = [1800.0, 2100.0]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, m, v in got:
        assert m == 2100.0                       # every rank sees the slowest rank's time
        assert v == pytest.approx(world * 1e3 / 2100.0)


def test_single_process_path_needs_no_group():
    import bench
    assert bench.max_over_ranks(12.5, None, torch.device("cpu")) == 12.5
    assert bench.replica_value(1, 500.0) == 2.0

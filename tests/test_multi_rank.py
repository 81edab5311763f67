"""Host logic of the N > 1 launch path, on CPU with gloo and world_size 2.

Each rank runs an independent acquisition; the whole-job value is the sum of
the ranks' units divided by the slowest rank's time (max over ranks)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 3.0][rank]               # the slower rank decides the job time
    value, t_max = bench.combine_ranks(seconds, 30, world)
    q.put((rank, value, t_max))
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t_max in out:
        assert t_max == pytest.approx(3.0)
        assert value == pytest.approx(2 * 30 / 3.0)


def test_single_rank_needs_no_process_group():
    import bench
    value, t_max = bench.combine_ranks(1.5, 30, 1)
    assert value == pytest.approx(20.0) and t_max == 1.5

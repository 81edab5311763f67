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


def _shard_worker(rank, world, port, q):
    """One rank of a patch-sharded iteration, computed by the FP64 oracle on this rank's
    patches with the two exchanges of the GPU path: the CMPE totals {sum |arg z|, M}
    after the forward pass, the gradient after the adjoint."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    import oracle
    import synth
    from paper_2608_06853_b300.shard import shard_problem
    p = synth.config_tiny(n_ang=3, n_rad=3, patch_w=3)
    psi = synth.simulate(p, 600, seed=31)
    s = 1.0 / (1530.0 + 20.0 * np.random.default_rng(2).standard_normal((p.nz, p.nx)))
    o = oracle.Oracle(shard_problem(p, rank, world))
    T, apod, phi = o.delays(s)
    B = o.das(psi, T, apod)
    L_loc, z, _, mask, M = o.cmpe(B)
    tot = torch.tensor([L_loc * max(M, 1), float(M)], dtype=torch.float64)
    dist.all_reduce(tot)
    m_all = int(round(float(tot[1])))
    G = o.cmpe_adjoint(B, z, mask, m_all)
    gT = o.das_adjoint(psi, T, apod, G)
    grad = torch.from_numpy(o.ray_adjoint(s, phi, apod, gT) + o.regularizer_grad(s))
    dist.all_reduce(grad)
    rtv, rsv = o.regularizers(s)
    L = float(tot[0]) / max(m_all, 1) + p.w1 * rtv + p.w2 * rsv
    q.put((rank, L, m_all, grad.numpy()))
    dist.destroy_process_group()


def test_patch_sharded_iteration_matches_single_rank_oracle():
    """Patches split over two gloo ranks (contiguous halves, regularisers on rank 0):
    after the exchange of the CMPE totals and of the gradient, every rank holds the loss
    and dL/ds of the whole problem, as the single-rank oracle computes them."""
    import numpy as np

    import oracle
    import synth
    from paper_2608_06853_b300.shard import patch_range, shard_problem
    assert [patch_range(9, r, 2) for r in range(2)] == [(0, 5), (5, 9)]
    assert [patch_range(10, r, 4) for r in range(4)] == [(0, 3), (3, 6), (6, 8), (8, 10)]
    p = synth.config_tiny(n_ang=3, n_rad=3, patch_w=3)
    assert shard_problem(p, 1, 2).w1 == 0.0 and shard_problem(p, 0, 2).w1 == p.w1
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    psi = synth.simulate(p, 600, seed=31)
    s = 1.0 / (1530.0 + 20.0 * np.random.default_rng(2).standard_normal((p.nz, p.nx)))
    parts, g, _, M = oracle.Oracle(p).loss_grad(psi, s)
    assert M > 0
    for rank, L, m_all, grad in out:
        assert m_all == M
        assert L == pytest.approx(parts[0], rel=1e-12)
        assert np.linalg.norm(grad - g) <= 1e-12 * np.linalg.norm(g)

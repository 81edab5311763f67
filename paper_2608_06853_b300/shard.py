"""One acquisition over several GPUs, split by patches.

The loss of Eq. 12 is a sum over patches (the CMPE term, Sec. II-D) plus the
regularisers of Eq. 10-11, and every patch's contribution to dL/ds depends on
the slowness map alone.  Each rank therefore plans the same array, grid and
channel data with a contiguous share of the patches; an iteration is

    af_forward (own patches) -> all-reduce of {sum |arg z|, M} (2 doubles) ->
    af_set_cmpe_totals -> af_adjoint -> all-reduce of dL/ds (nz * nx floats) ->
    af_step (the same update on every rank)

with the regularisers given to rank 0 only.  The library does the arithmetic;
this module only splits the problem and issues the two collectives
(torch.distributed: NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

import dataclasses

import numpy as np


def patch_range(n_patch: int, rank: int, world: int):
    """Contiguous patches [lo, hi) of rank `rank` out of `world` (sizes differ by <= 1)."""
    base, extra = divmod(n_patch, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_problem(problem, rank: int, world: int):
    """The problem restricted to this rank's patches; the regularisers stay on rank 0."""
    lo, hi = patch_range(problem.n_patch, rank, world)
    npx = problem.patch_npix
    over = dict(n_patch=hi - lo, pix_x=np.asarray(problem.pix_x)[lo * npx:hi * npx],
                pix_z=np.asarray(problem.pix_z)[lo * npx:hi * npx])
    if rank != 0:
        over.update(w1=0.0, w2=0.0)
    return dataclasses.replace(problem, **over)


class ShardedPlan:
    """A rank's plan of a patch-sharded problem and its iteration with the two
    all-reduces.  `group` is a torch.distributed process group (None: default)."""

    def __init__(self, problem, rank: int, world: int, iq_dtype: int = 0, stream=None, group=None):
        from . import Plan
        self.problem = problem
        self.rank, self.world, self.group = rank, world, group
        self.plan = Plan(shard_problem(problem, rank, world), iq_dtype=iq_dtype, stream=stream)

    def iterate(self, iq, s, grad, m, v, step: int, loss, iq_scale=None):
        """One iteration of the whole problem; afterwards s, m, v, grad and loss are the
        same on every rank."""
        import torch
        import torch.distributed as dist
        pl = self.plan
        with torch.cuda.stream(pl.stream):
            pl.af_forward(iq, s, loss, iq_scale)
            tot = pl.cmpe_totals()
            if self.world > 1:
                dist.all_reduce(tot, group=self.group)
            pl.set_cmpe_totals(tot, loss)
            pl.af_adjoint(grad)
            if self.world > 1:
                dist.all_reduce(grad, group=self.group)
            if self.rank != 0:
                # every plan computes R_TV and R_SV; only rank 0 weighs them into its loss
                loss[0:1] = loss[1:2] + self.problem.w1 * loss[2:3] + self.problem.w2 * loss[3:4]
            pl.af_step(grad, s, m, v, step)

    def close(self):
        self.plan.close()

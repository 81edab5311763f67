"""Batched autofocus of independent acquisitions as one CUDA graph.

Each acquisition has its own plan (af_plan) and stream.  `BatchRunner.capture`
records `iterations` calls of af_iterate for every acquisition, each on its
own stream forked from and joined back to a capture stream, into one CUDA
graph; `replay()` then runs the whole job (all acquisitions, all iterations)
with a single graph launch.  The af_* calls of an iteration allocate nothing
and never synchronise, so they are capturable; the Adam step index is a
launch argument and is captured per iteration.  This module only sequences
calls: every step of the computation runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import Plan


class BatchRunner:
    def __init__(self, problems, iqs, scales=None, iq_dtype=0, device=None):
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(device=self.device) for _ in problems]
        self.plans = [Plan(p, iq_dtype=iq_dtype, stream=st) for p, st in zip(problems, self.streams)]
        self.problems = list(problems)
        self.iqs = list(iqs)
        self.scales = list(scales) if scales is not None else [None] * len(problems)
        self.s0 = [torch.from_numpy(p.initial_slowness()).to(self.device) for p in problems]
        self.s = [x.clone() for x in self.s0]
        self.m = [torch.zeros_like(x) for x in self.s0]
        self.v = [torch.zeros_like(x) for x in self.s0]
        self.g = [torch.zeros_like(x) for x in self.s0]
        self.loss = [torch.zeros(4, device=self.device) for _ in problems]
        self.graph = None

    def reset(self):
        """Initial slowness and zero Adam moments (outside the graph)."""
        for k in range(len(self.plans)):
            self.s[k].copy_(self.s0[k])
            self.m[k].zero_()
            self.v[k].zero_()
        torch.cuda.synchronize(self.device)

    def _issue(self, iterations, first_step=1):
        for k, plan in enumerate(self.plans):
            with torch.cuda.stream(self.streams[k]):
                for it in range(first_step, first_step + iterations):
                    plan.af_iterate(self.iqs[k], self.s[k], self.g[k], self.m[k], self.v[k], it, self.loss[k],
                                    self.scales[k])

    def run_eager(self, iterations):
        """The same calls without a graph, stream by stream."""
        cur = torch.cuda.current_stream(self.device)
        for st in self.streams:
            st.wait_stream(cur)
        self._issue(iterations)
        for st in self.streams:
            cur.wait_stream(st)

    def capture(self, iterations, warmup=True):
        """Record `iterations` autofocus iterations of every acquisition into one graph."""
        if warmup:                                   # first calls set up warm starts outside capture
            self.run_eager(1)
            torch.cuda.synchronize(self.device)
            self.reset()
        self.graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=self.device)
        cap.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.graph(self.graph, stream=cap):
            for st in self.streams:
                st.wait_stream(cap)
            self._issue(iterations)
            for st in self.streams:
                cap.wait_stream(st)
        torch.cuda.synchronize(self.device)
        return self.graph

    def replay(self):
        self.graph.replay()

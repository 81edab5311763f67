"""Batched autofocus of independent acquisitions as one CUDA graph.

A thin binding of the batch calls of the C ABI (af_batch_plan, af_batch_iterate,
af_batch_capture, af_batch_launch): the library owns one plan and one stream per
acquisition, forks them from the caller's stream and joins them back.
`BatchRunner.capture` records `iterations` calls of af_iterate for every
acquisition into one CUDA graph; `replay()` runs the whole job (all
acquisitions, all iterations) with a single graph launch.  This module only
marshals arguments: every step of the computation runs in the library's
kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import AfConfig, Plan, _check, iq_view, load, make_config


def _array(tensors):
    """Host array of the tensors' device pointers (NULL for None)."""
    out = (ctypes.c_void_p * len(tensors))()
    for k, t in enumerate(tensors):
        if t is not None:
            if not t.is_cuda or not t.is_contiguous():
                raise ValueError("contiguous device tensors only")
            out[k] = t.data_ptr()
    return out


class BatchRunner:
    def __init__(self, problems, iqs, scales=None, iq_dtype=0, device=None, stream=None):
        self.lib = load()
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.problems = list(problems)
        n = len(self.problems)
        cfgs = [make_config(p, iq_dtype) for p in self.problems]     # (config, kept arrays)
        self._cfgs = cfgs
        cfg_ptrs = (ctypes.POINTER(AfConfig) * n)(*[ctypes.pointer(c) for c, _ in cfgs])
        h = ctypes.c_void_p()
        _check(self.lib.af_batch_plan(n, cfg_ptrs, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
               "af_batch_plan")
        self.handle = h
        self.plans = [Plan.batch_member(self, k, p, iq_dtype, self.stream) for k, p in enumerate(self.problems)]
        self.iqs = [iq_view(x) for x in iqs]
        self.scales = list(scales) if scales is not None else [None] * n
        with torch.cuda.stream(self.stream):
            self.s0 = [torch.from_numpy(p.initial_slowness()).to(self.device) for p in self.problems]
            self.s = [x.clone() for x in self.s0]
            self.m = [torch.zeros_like(x) for x in self.s0]
            self.v = [torch.zeros_like(x) for x in self.s0]
            self.g = [torch.zeros_like(x) for x in self.s0]
            self.loss = [torch.zeros(4, device=self.device) for _ in self.problems]
        self._ptrs = [_array(x) for x in (self.iqs, self.scales, self.s, self.g, self.m, self.v, self.loss)]
        self.captured = False

    def reset(self):
        """Initial slowness and zero Adam moments (outside the graph)."""
        with torch.cuda.stream(self.stream):
            for k in range(len(self.problems)):
                self.s[k].copy_(self.s0[k])
                self.m[k].zero_()
                self.v[k].zero_()
        torch.cuda.synchronize(self.device)

    def run_eager(self, iterations, first_step=1):
        """The same calls without a graph: one af_batch_iterate per iteration."""
        iq, sc, s, g, m, v, loss = self._ptrs
        for it in range(first_step, first_step + iterations):
            _check(self.lib.af_batch_iterate(self.handle, iq, sc, s, g, m, v, int(it), loss), "af_batch_iterate")

    def capture(self, iterations, warmup=True, first_step=1):
        """Record `iterations` autofocus iterations of every acquisition into one graph."""
        if warmup:                                   # first calls set up warm starts outside capture
            self.run_eager(1)
            torch.cuda.synchronize(self.device)
            self.reset()
        iq, sc, s, g, m, v, loss = self._ptrs
        _check(self.lib.af_batch_capture(self.handle, iq, sc, s, g, m, v, loss, int(first_step), int(iterations)),
               "af_batch_capture")
        self.captured = True

    def replay(self):
        _check(self.lib.af_batch_launch(self.handle), "af_batch_launch")

    def close(self):
        if getattr(self, "handle", None):
            for p in self.plans:
                p.handle = None
            self.lib.af_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

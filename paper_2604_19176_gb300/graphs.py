"""CUDA-graph capture of operator calls on fixed buffers.

A plan's kernels allocate nothing and synchronise nothing while they run, and
their work queues re-arm themselves at the end of each launch, so a sequence
of operator calls on fixed device buffers can be captured once into a CUDA
graph and replayed with a single launch.  :class:`GraphedOperator` does this
for the batched forward + adjoint of a multi-instance plan (uneven geometries
in one plan: every kernel is persistent and walks all instances' work), and
for the fused TV iteration.
"""
from __future__ import annotations

import torch

from .api import PatPlan

__all__ = ["GraphedOperator", "GraphedTVStep"]


class GraphedOperator:
    """g_out = A f_in and f_out = A^T g_in, replayed from one CUDA graph.

    Fill ``f_in`` / ``g_in`` in place and call :meth:`replay`; results appear
    in ``g_out`` / ``f_out``.
    """

    def __init__(self, plan: PatPlan, forward: bool = True, adjoint: bool = True, warmup: int = 2):
        if not (forward or adjoint):
            raise ValueError("nothing to capture")
        self.plan = plan
        dev = plan.device
        self.f_in = torch.zeros(plan.image_shape(), dtype=plan.image_dtype, device=dev)
        self.g_in = torch.zeros(plan.data_shape(), dtype=torch.float32, device=dev)
        self.g_out = torch.zeros(plan.data_shape(), dtype=torch.float32, device=dev)
        self.f_out = torch.zeros(plan.image_shape(), dtype=plan.image_dtype, device=dev)
        self._fwd, self._adj = forward, adjoint
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self._body(side)
        torch.cuda.current_stream(dev).wait_stream(side)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body(torch.cuda.current_stream(dev))

    def _body(self, stream) -> None:
        if self._fwd:
            self.plan.forward(self.f_in, out=self.g_out, stream=stream)
        if self._adj:
            self.plan.adjoint(self.g_in, out=self.f_out, stream=stream)

    def replay(self) -> None:
        self.graph.replay()


class GraphedTVStep:
    """Two fused TV iterations (f_a -> f_b -> f_a) replayed from one graph."""

    def __init__(self, plan: PatPlan, g: torch.Tensor, tau: float, lam: float, eps: float, nonneg: bool = True):
        self.plan = plan
        dev = plan.device
        self.g = g
        self.f = torch.zeros(plan.image_shape(), dtype=torch.float32, device=dev)
        self._tmp = torch.zeros_like(self.f)
        self.args = (tau, lam, eps, nonneg)
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self._body(side)
        torch.cuda.current_stream(dev).wait_stream(side)
        self.f.zero_()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body(torch.cuda.current_stream(dev))

    def _body(self, stream) -> None:
        tau, lam, eps, nonneg = self.args
        self.plan.tv_step(self.f, self._tmp, self.g, tau, lam, eps, nonneg=nonneg, stream=stream)
        self.plan.tv_step(self._tmp, self.f, self.g, tau, lam, eps, nonneg=nonneg, stream=stream)

    def replay(self) -> None:
        self.graph.replay()

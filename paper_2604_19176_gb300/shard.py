"""Multi-GPU partitioning of the operators: one process (rank) per GPU.

Two splits, both exact rearrangements of the single-GPU operators:

* **Instances.**  The instances of a batch are independent problems (every
  operator acts on each instance alone), so a rank owns a plan of some of
  them and no data moves between ranks.  :func:`lpt_assign` balances the
  ranks by each instance's cost (its samples per operator call) with the
  longest-processing-time rule; :class:`InstanceShard` holds a rank's plan
  and gathers per-instance results to one rank only when asked.

* **Detectors of one instance.**  A's rows are detectors, so A = [A_1; ...;
  A_R] for contiguous detector ranges, and A^T g = sum_r A_r^T g_r.  A
  contiguous run of detectors j0 .. j0 + s - 1 of an arc is itself an arc
  (start theta0 + j0 Phi / n_det, span s Phi / n_det, s detectors) with the
  same detector angles, so rank r's plan is an ordinary plan of its sub-arc.
  The forward needs no exchange (each rank computes its rows); the adjoint
  needs one all-reduce (sum) of the N x N partial images.  This is the split
  for a single large image, e.g. the 760 x 760, 256-detector experimental
  geometry of Sec. 2.4.2.

The per-rank operator is a :class:`~paper_2604_19176_gb300.api.PatPlan` by
default; ``make_op`` replaces it (any object with ``forward(f)`` and
``adjoint(g)`` over torch tensors), which is how the CPU tests run the
partition logic with gloo ranks.  Collectives go through
``torch.distributed`` (NCCL on GPUs); nothing here uses a multicast or peer
mapping.
"""
from __future__ import annotations

import heapq
from typing import Callable, Optional, Sequence

import torch

from .api import Geometry, PatPlan

__all__ = ["lpt_assign", "detector_ranges", "sub_arc", "instance_cost", "InstanceShard", "DetectorShard"]


def instance_cost(g: Geometry) -> float:
    """Cost proxy of one instance: its (detector, radius, angle) sample count
    bound n_det (n_t + 2) K (the circular means and their adjoint dominate)."""
    return float(g.n_det) * (g.n_t + 2) * g.n_angles


def lpt_assign(costs: Sequence[float], world: int) -> list[list[int]]:
    """Instances per rank by the longest-processing-time rule: instances in
    decreasing cost, each to the currently least loaded rank (ties to the
    lower rank).  Every instance goes to exactly one rank; a rank's list is
    in increasing instance order.  Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(x) for x in out]


def detector_ranges(n_det: int, world: int) -> list[tuple[int, int]]:
    """Contiguous detector ranges (j0, count), as equal as possible, in rank
    order; requires n_det >= world."""
    if world < 1 or n_det < world:
        raise ValueError("need 1 <= world <= n_det")
    edges = [(r * n_det) // world for r in range(world + 1)]
    return [(edges[r], edges[r + 1] - edges[r]) for r in range(world)]


def sub_arc(g: Geometry, j0: int, count: int) -> Geometry:
    """The arc of detectors j0 .. j0 + count - 1 of g (same angles, time grid
    and angular rule)."""
    if not (0 <= j0 and count >= 1 and j0 + count <= g.n_det):
        raise ValueError("detector range outside the geometry")
    step = g.arc_span / g.n_det
    return Geometry(g.n, count, g.arc_start + j0 * step, count * step, g.n_t, g.t_max, g.n_angles)


def _default_op(geoms, device):
    return PatPlan(list(geoms), device=device, tune=1)


class InstanceShard:
    """A rank's share of a batch of instances (no exchange on the data path).

    geoms:  all instances of the batch (every rank passes the same list).
    make_op(geoms, device): builds the rank's operator over its instances.
    The rank's operator sees its instances packed in increasing instance
    order (``self.mine``).
    """

    def __init__(self, geoms: Sequence[Geometry], rank: int, world: int, *, device=None,
                 make_op: Optional[Callable] = None, costs: Optional[Sequence[float]] = None):
        self.geoms = list(geoms)
        self.rank, self.world = rank, world
        self.assign = lpt_assign(costs if costs is not None else [instance_cost(g) for g in self.geoms], world)
        self.mine = self.assign[rank]
        self.op = (make_op or _default_op)([self.geoms[i] for i in self.mine], device) if self.mine else None

    def forward(self, f):
        return self.op.forward(f) if self.op is not None else None

    def adjoint(self, g):
        return self.op.adjoint(g) if self.op is not None else None

    def gather(self, local: Sequence[torch.Tensor], dst: int = 0) -> Optional[list]:
        """Per-instance results (``local[k]`` belongs to instance
        ``self.mine[k]``) collected on rank ``dst`` in instance order; other
        ranks get None.  Uses object gathering (host copies), meant for final
        results, not for the iteration loop."""
        import torch.distributed as dist

        payload = [(i, t.detach().cpu()) for i, t in zip(self.mine, local)]
        if self.world == 1:
            return [t for _, t in sorted(payload, key=lambda x: x[0])]
        bucket = [None] * self.world if self.rank == dst else None
        dist.gather_object(payload, bucket, dst=dst)
        if self.rank != dst:
            return None
        out = [None] * len(self.geoms)
        for part in bucket:
            for i, t in part:
                out[i] = t
        return out


class DetectorShard:
    """A rank's detector sub-arc of one instance.

    forward(f) -> this rank's rows of A f (count x n_t);
    adjoint(g_rows) -> the full A^T g (N x N) on every rank: the rank's
    partial A_r^T g_r plus one all-reduce (sum) over the process group;
    gather_rows(rows) -> the full n_det x n_t data on every rank.
    """

    def __init__(self, g: Geometry, rank: int, world: int, *, device=None, make_op: Optional[Callable] = None,
                 group=None):
        self.g = g
        self.rank, self.world = rank, world
        self.group = group
        self.ranges = detector_ranges(g.n_det, world)
        self.j0, self.count = self.ranges[rank]
        self.sub = sub_arc(g, self.j0, self.count)
        self.op = (make_op or _default_op)([self.sub], device)

    def forward(self, f: torch.Tensor) -> torch.Tensor:
        return self.op.forward(f)

    def adjoint(self, g_rows: torch.Tensor) -> torch.Tensor:
        part = self.op.adjoint(g_rows)
        if self.world > 1:
            import torch.distributed as dist

            dist.all_reduce(part, op=dist.ReduceOp.SUM, group=self.group)
        return part

    def gather_rows(self, rows: torch.Tensor) -> torch.Tensor:
        if self.world == 1:
            return rows
        import torch.distributed as dist

        pieces = [torch.empty((c, self.g.n_t), dtype=rows.dtype, device=rows.device) for _, c in self.ranges]
        # all_gather needs equal shapes: pad every piece to the largest count
        cmax = max(c for _, c in self.ranges)
        buf = torch.zeros((cmax, self.g.n_t), dtype=rows.dtype, device=rows.device)
        buf[: self.count] = rows
        bufs = [torch.empty_like(buf) for _ in range(self.world)]
        dist.all_gather(bufs, buf, group=self.group)
        for r, (_, c) in enumerate(self.ranges):
            pieces[r] = bufs[r][:c]
        return torch.cat(pieces, dim=0)

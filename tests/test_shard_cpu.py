"""Multi-GPU partitioning (paper_2604_19176_gb300.shard) with two gloo ranks on CPU.

The per-rank operator is the FP64 oracle here (the product uses a PatPlan per
rank); the tests check the partition logic itself:
  - instances split by LPT, each rank applies A to its own instances, the
    results gathered on rank 0 equal the single-rank results;
  - one instance split by detectors: the ranks' rows of A f, gathered, equal
    A f of the whole arc, and the all-reduced sum of the ranks' partial
    adjoints equals A^T g of the whole arc (to FP64 rounding: the sub-arc
    angles are recomputed from the arc's start and span).
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
from paper_2604_19176_gb300 import Geometry, inputs
from paper_2604_19176_gb300.shard import detector_ranges, instance_cost, lpt_assign, sub_arc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

GEOMS = [Geometry(16, 6, 0.0, 2 * math.pi, 12, 2.0, 16), Geometry(24, 9, 0.4, math.pi, 20, 2.0, 24),
         Geometry(12, 5, 1.0, 1.5 * math.pi, 10, 2.5, 12), Geometry(20, 7, -0.3, 0.8 * math.pi, 16, 2.0, 20),
         Geometry(16, 4, 0.0, math.pi, 8, 2.0, 16)]
SPLIT = Geometry(24, 11, 0.3, 1.7 * math.pi, 18, 2.0, 28)


def og(g):
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


class OracleOp:
    """forward / adjoint of a list of instances, packed like a plan's buffers."""

    def __init__(self, geoms, device=None):
        self.geoms = list(geoms)

    def forward(self, f):
        out, o = [], 0
        for g in self.geoms:
            out.append(torch.tensor(O.forward(og(g), f[o:o + g.n * g.n].reshape(g.n, g.n).numpy()).ravel()))
            o += g.n * g.n
        return torch.cat(out)

    def adjoint(self, d):
        out, o = [], 0
        for g in self.geoms:
            k = g.n_det * g.n_t
            out.append(torch.tensor(O.adjoint(og(g), d[o:o + k].reshape(g.n_det, g.n_t).numpy()).ravel()))
            o += k
        return torch.cat(out)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    import sys

    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    from paper_2604_19176_gb300.shard import DetectorShard, InstanceShard
    from test_shard_cpu import GEOMS, SPLIT, OracleOp

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # instances
        sh = InstanceShard(GEOMS, rank, world, make_op=OracleOp)
        packed = torch.cat([torch.tensor(inputs.random_image(GEOMS[i].n, seed=100 + i)).ravel() for i in sh.mine])
        out = sh.forward(packed)          # the rank's instances, packed in instance order
        sizes = [GEOMS[i].n_det * GEOMS[i].n_t for i in sh.mine]
        got = sh.gather(list(torch.split(out, sizes)), dst=0)
        if rank == 0:
            np.savez(os.path.join(out_dir, "inst.npz"), *[t.numpy() for t in got])
        # detectors of one instance
        ds = DetectorShard(SPLIT, rank, world, make_op=OracleOp)
        f = torch.tensor(inputs.random_image(SPLIT.n, seed=7)).ravel()
        rows = ds.forward(f).reshape(ds.count, SPLIT.n_t)
        full = ds.gather_rows(rows)
        d = torch.tensor(inputs.random_data(SPLIT.n_det, SPLIT.n_t, seed=8))
        adj = ds.adjoint(d[ds.j0:ds.j0 + ds.count].reshape(-1).clone())
        np.save(os.path.join(out_dir, f"det_fwd{rank}.npy"), full.numpy())
        np.save(os.path.join(out_dir, f"det_adj{rank}.npy"), adj.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_lpt_assign_balances_and_covers():
    costs = [9, 7, 6, 5, 4, 3, 2, 2, 1]
    a = lpt_assign(costs, 3)
    assert sorted(i for r in a for i in r) == list(range(len(costs)))
    loads = [sum(costs[i] for i in r) for r in a]
    assert max(loads) - min(loads) <= max(costs)        # the LPT bound
    assert a == lpt_assign(costs, 3)                     # deterministic
    assert lpt_assign([1.0], 4) == [[0], [], [], []]
    assert instance_cost(GEOMS[0]) == 6 * 14 * 16


def test_detector_ranges_and_sub_arc_keep_the_angles():
    assert detector_ranges(11, 2) == [(0, 5), (5, 6)]
    assert detector_ranges(8, 4) == [(0, 2), (2, 2), (4, 2), (6, 2)]
    with pytest.raises(ValueError):
        detector_ranges(2, 3)
    g = SPLIT
    full = O.detectors(og(g))
    for j0, c in detector_ranges(g.n_det, 3):
        np.testing.assert_allclose(O.detectors(og(sub_arc(g, j0, c))), full[j0:j0 + c], rtol=0, atol=1e-14)


def test_two_gloo_ranks_reproduce_the_single_rank_operators(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "inst.npz")
    for i, g in enumerate(GEOMS):
        ref = O.forward(og(g), inputs.random_image(g.n, seed=100 + i)).ravel()
        np.testing.assert_array_equal(got[f"arr_{i}"], ref)
    ref_f = O.forward(og(SPLIT), inputs.random_image(SPLIT.n, seed=7))
    ref_a = O.adjoint(og(SPLIT), inputs.random_data(SPLIT.n_det, SPLIT.n_t, seed=8))
    for r in range(world):
        f_r = np.load(tmp_path / f"det_fwd{r}.npy")
        a_r = np.load(tmp_path / f"det_adj{r}.npy").reshape(SPLIT.n, SPLIT.n)
        assert np.linalg.norm(f_r - ref_f) <= 1e-12 * np.linalg.norm(ref_f)
        assert np.linalg.norm(a_r - ref_a) <= 1e-12 * np.linalg.norm(ref_a)

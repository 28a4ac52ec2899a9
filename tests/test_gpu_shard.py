"""The detector split of one instance (paper_2604_19176_gb300.shard) on one GPU.

One process holds the plans of two detector sub-arcs of one geometry on the
same device (the two ranks' plans, without the process group): the sub-arcs'
rows of A f, stacked, and the sum of their partial adjoints (the all-reduce,
done here on the host) match the FP64 oracle of the whole arc within the
FP32 tolerance.  The same through InstanceShard / DetectorShard with one rank.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_19176_gb300 import Geometry, PatPlan, inputs
from paper_2604_19176_gb300.shard import DetectorShard, InstanceShard, detector_ranges, sub_arc

pytestmark = pytest.mark.gpu

TOL = 1e-5


def og(g):
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("parts", [2, 3])
def test_subarc_plans_reproduce_the_whole_operator(cuda_dev, parts):
    g = Geometry(128, 40, 0.2, 1.5 * math.pi, 160, 2.0, 256)
    f_np = inputs.random_image(128, seed=51).astype(np.float32)
    d_np = inputs.random_data(40, 160, seed=52).astype(np.float32)
    f = torch.tensor(f_np, device=cuda_dev)
    rows, adj = [], torch.zeros(128, 128, dtype=torch.float64, device=cuda_dev)
    for j0, c in detector_ranges(g.n_det, parts):
        p = PatPlan(sub_arc(g, j0, c), device=cuda_dev)
        rows.append(p.forward(f).double())
        adj += p.adjoint(torch.tensor(d_np[j0:j0 + c], device=cuda_dev)).double()
        p.close()
    torch.cuda.synchronize()
    ref_g = O.forward(og(g), f_np.astype(np.float64))
    ref_f = O.adjoint(og(g), d_np.astype(np.float64))
    assert rel(torch.cat(rows).cpu().numpy(), ref_g) <= TOL
    assert rel(adj.cpu().numpy(), ref_f) <= TOL


def test_shard_classes_with_one_rank(cuda_dev):
    geoms = [Geometry(64, 16, 0.0, math.pi, 48, 2.0, 64), Geometry(48, 12, 0.5, 2 * math.pi, 40, 2.0, 96)]
    sh = InstanceShard(geoms, 0, 1, device=cuda_dev)
    assert sh.mine == [0, 1]
    imgs = [inputs.random_image(g.n, seed=60 + i).astype(np.float32) for i, g in enumerate(geoms)]
    out = sh.forward(torch.tensor(np.concatenate([x.ravel() for x in imgs]), device=cuda_dev))
    fo, go = sh.op.layout()
    got = sh.gather([out[go[k]:go[k + 1]] for k in range(len(geoms))])
    for i, g in enumerate(geoms):
        assert rel(got[i].double().numpy().reshape(g.n_det, g.n_t), O.forward(og(g), imgs[i].astype(np.float64))) <= TOL
    g = geoms[1]
    ds = DetectorShard(g, 0, 1, device=cuda_dev)
    d = inputs.random_data(g.n_det, g.n_t, seed=62).astype(np.float32)
    a = ds.adjoint(torch.tensor(d, device=cuda_dev)).double().cpu().numpy()
    assert rel(a, O.adjoint(og(g), d.astype(np.float64))) <= TOL

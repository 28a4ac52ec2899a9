"""GPU approximate inverses for the DIP input (Sec. 2.2) against the FP64
oracle's iterations (``oracle/inverse.py``) on the oracle's A.

Tolerance: A and A^T meet 1e-5 relative L2 per application.  Landweber with
omega <= 1/||A||^2 is non-expansive, so k steps stay within k * 1e-5.  CGLS
is not non-expansive; its step lengths are ratios of inner products that
FP32 operators perturb at the same 1e-5 level, and at 6 steps on this
geometry the bound taken is 10x the Landweber one.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import inverse as OI
from paper_2604_19176_gb300 import Geometry, PatPlan, inputs
from paper_2604_19176_gb300.recon import UNet, dip_reconstruct, initial_reconstruction

pytestmark = pytest.mark.gpu


def og(g):
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def _setup(cuda_dev, geoms):
    plan = PatPlan(geoms, device=cuda_dev)
    datas = []
    for i, g in enumerate(geoms):
        f = inputs.vessel_phantom(g.n, seed=20 + i)
        datas.append(inputs.add_noise(O.forward(og(g), f), 0.02, seed=30 + i).astype(np.float32).astype(np.float64))
    gd = torch.tensor(np.concatenate([d.ravel() for d in datas]), dtype=torch.float32, device=cuda_dev)
    return plan, datas, gd.reshape(plan.data_shape())


def test_landweber_matches_oracle(cuda_dev):
    g = Geometry(64, 48, 0.3, 1.5 * math.pi, 96, 2.0, 128)
    plan, datas, gd = _setup(cuda_dev, [g])
    k, omega = 10, 1.0
    f = initial_reconstruction(plan, gd, "landweber", iters=k, omega=omega)
    ref = OI.landweber(lambda x: O.forward(og(g), x), lambda y: O.adjoint(og(g), y), datas[0], (g.n, g.n), omega, k)
    assert rel(f.double().cpu().numpy(), ref) <= k * 1e-5


def test_cgls_matches_oracle_per_instance(cuda_dev):
    """Two uneven instances in one plan: CGLS step lengths are per instance, so
    each instance follows the oracle's CGLS on that instance alone."""
    geoms = [Geometry(64, 48, 0.3, 1.5 * math.pi, 96, 2.0, 128), Geometry(48, 40, 1.0, math.pi, 80, 2.0, 96)]
    plan, datas, gd = _setup(cuda_dev, geoms)
    k = 6
    f = initial_reconstruction(plan, gd, "cgls", iters=k).double().cpu().numpy().ravel()
    fo, _ = plan.layout()
    for i, g in enumerate(geoms):
        ref, res = OI.cgls(lambda x: O.forward(og(g), x), lambda y: O.adjoint(og(g), y), datas[i], (g.n, g.n), k)
        assert res[-1] < 0.5 * res[0]
        assert rel(f[fo[i]:fo[i + 1]].reshape(g.n, g.n), ref) <= 10 * k * 1e-5


def test_dip_from_initial_reconstruction(cuda_dev):
    """The DIP loop with the approximate inverse as its one-channel input
    instead of noise (Sec. 2.2), and the mouse-data head and penalty."""
    g = Geometry(32, 32, 0.0, 1.5 * math.pi, 48, 2.0, 64)
    plan, datas, gd = _setup(cuda_dev, [g])
    z = initial_reconstruction(plan, gd, "cgls", iters=5).reshape(1, 1, g.n, g.n)
    torch.manual_seed(0)
    net = UNet(in_ch=1, base=8, mouse=True).to(cuda_dev)
    f, hist, _ = dip_reconstruct(plan, gd, z, lam=1e-4, steps=20, lr=1e-3, cosine=True, net=net,
                                 callback=lambda *a: None, mean_penalty=(1.0, 0.1))
    assert torch.isfinite(f).all() and hist[-1] < hist[0]

"""The fused time stage of pat_tv_step / pat_pdhg_step (k_time_pair).

One launch per step replaces the radius sums of the circular means, the
forward Abel stage with the residual (or the dual update), and the adjoint
Abel stage; a thread-block cluster owns 4 detectors' rows.  Checked here:
  - the TV step through the fused stage against the FP64 oracle of
    f - tau (A^T (A f - g) + lam grad TV_eps(f)), relative to the update;
  - the primal-dual step's dual variable y = sigma (A fbar - g) / (1 + sigma)
    from y = 0 against the oracle's A;
  - fused and separate plans (time_pair = 0 / 1) agree to FP32 summation
    order, on detector counts that leave a partial group, time axes shorter
    than one chunk per cluster CTA, a 2048-sample time axis, and an uneven
    batch;
  - a time axis too long for the fused stage's shared memory falls back to the
    separate launches (plan info time_pair = 0).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_19176_gb300 import Geometry, PatPlan, inputs

pytestmark = pytest.mark.gpu


def og(g):
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_tv_step_through_the_fused_stage_matches_the_oracle(cuda_dev):
    g = Geometry(64, 29, 0.3, 1.1 * math.pi, 112, 2.0, 128)
    plan = PatPlan(g, device=cuda_dev)
    assert plan.info()["time_pair"] == 1
    f_np = f32(np.abs(inputs.random_image(64, seed=71)))
    d_np = f32(inputs.random_data(29, 112, seed=72))
    tau, lam, eps = 0.5, 0.05, 1e-2
    out = torch.empty(64, 64, device=cuda_dev)
    plan.tv_step(torch.tensor(f_np, dtype=torch.float32, device=cuda_dev), out,
                 torch.tensor(d_np, dtype=torch.float32, device=cuda_dev), tau, lam, eps, nonneg=False)
    torch.cuda.synchronize()
    r = O.forward(og(g), f_np) - d_np
    _, tvg = O.tv(f_np, eps)
    ref = f_np - tau * (O.adjoint(og(g), r) + lam * tvg)
    # the FP32 operators meet 1e-5 of A^T r; the update is measured against its own size
    assert rel(out.double().cpu().numpy() - f_np, ref - f_np) <= 2e-5


def test_pdhg_dual_update_through_the_fused_stage(cuda_dev):
    g = Geometry(48, 21, -0.2, 1.4 * math.pi, 70, 2.0, 96)
    plan = PatPlan(g, device=cuda_dev)
    assert plan.info()["time_pair"] == 1
    fb = f32(np.abs(inputs.random_image(48, seed=73)))
    d_np = f32(inputs.random_data(21, 70, seed=74))
    z = lambda s: torch.zeros(s, dtype=torch.float32, device=cuda_dev)  # noqa: E731
    f, px, py, y = z((48, 48)), z((48, 48)), z((48, 48)), z((21, 70))
    fbar = torch.tensor(fb, dtype=torch.float32, device=cuda_dev)
    sigma = 0.7
    plan.pdhg_step(f, fbar, y, px, py, torch.tensor(d_np, dtype=torch.float32, device=cuda_dev), sigma, 0.1, 1e-3,
                   nonneg=False)
    torch.cuda.synchronize()
    ref = sigma * (O.forward(og(g), fb) - d_np) / (1.0 + sigma)
    assert rel(y.double().cpu().numpy(), ref) <= 1e-5


GEOMS = {
    "partial_group": [Geometry(64, 13, 0.1, math.pi, 96, 2.0, 128)],
    "short_time_axis": [Geometry(32, 11, 0.0, 2 * math.pi, 20, 2.0, 64)],
    "one_chunk_per_rank": [Geometry(48, 8, 0.4, math.pi, 250, 2.0, 64)],
    "time_axis_2048": [Geometry(128, 10, 0.0, math.pi, 2048, 2.0, 64)],
    "uneven_batch": [Geometry(64, 16, 0.0, math.pi, 96, 2.0, 128), Geometry(32, 9, 0.5, 1.5 * math.pi, 40, 2.0, 64),
                     Geometry(48, 24, -0.3, math.pi, 300, 2.5, 96)],
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_fused_and_separate_time_stages_agree(cuda_dev, name):
    geoms = GEOMS[name]
    fused = PatPlan(geoms, device=cuda_dev)
    sep = PatPlan(geoms, device=cuda_dev, time_pair=1)
    assert fused.info()["time_pair"] == 1 and sep.info()["time_pair"] == 0
    fe, ge = fused.f_elems, fused.g_elems
    rng = np.random.default_rng(75)
    f0 = torch.tensor(np.abs(rng.standard_normal(fe)), dtype=torch.float32, device=cuda_dev)
    d = torch.tensor(rng.standard_normal(ge), dtype=torch.float32, device=cuda_dev)
    shape_f, shape_g = fused.image_shape(), fused.data_shape()
    f0, d = f0.reshape(shape_f), d.reshape(shape_g)
    outs = []
    for p in (fused, sep):
        o = torch.empty_like(f0)
        p.tv_step(f0, o, d, 0.3, 0.05, 1e-2, nonneg=False)
        outs.append(o)
    torch.cuda.synchronize()
    assert rel(outs[0].double().cpu().numpy() - f0.double().cpu().numpy(),
               outs[1].double().cpu().numpy() - f0.double().cpu().numpy()) <= 2e-6
    ys = []
    for p in (fused, sep):
        z = lambda s: torch.zeros(s, dtype=torch.float32, device=cuda_dev)  # noqa: E731
        st = {"f": f0.clone(), "fbar": f0.clone(), "y": z(shape_g), "px": z(shape_f), "py": z(shape_f)}
        for _ in range(2):
            p.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], d, 0.5, 0.5, 1e-3, nonneg=False)
        ys.append(st)
    torch.cuda.synchronize()
    for k in ("f", "y"):
        assert rel(ys[0][k].double().cpu().numpy(), ys[1][k].double().cpu().numpy()) <= 2e-6


def test_fused_stage_is_deterministic(cuda_dev):
    g = Geometry(64, 40, 0.0, math.pi, 160, 2.0, 128)
    plan = PatPlan(g, device=cuda_dev)
    f0 = torch.tensor(np.abs(inputs.random_image(64, seed=76)), dtype=torch.float32, device=cuda_dev)
    d = torch.tensor(inputs.random_data(40, 160, seed=77), dtype=torch.float32, device=cuda_dev)
    a, b = torch.empty_like(f0), torch.empty_like(f0)
    plan.tv_step(f0, a, d, 0.3, 0.05, 1e-2)
    plan.tv_step(f0, b, d, 0.3, 0.05, 1e-2)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_long_time_axis_falls_back_to_separate_launches(cuda_dev):
    g = Geometry(32, 6, 0.0, math.pi, 6000, 2.0, 32)
    plan = PatPlan(g, device=cuda_dev)
    assert plan.info()["time_pair"] == 0
    f_np = f32(np.abs(inputs.random_image(32, seed=78)))
    d_np = f32(inputs.random_data(6, 6000, seed=79))
    out = torch.empty(32, 32, device=cuda_dev)
    plan.tv_step(torch.tensor(f_np, dtype=torch.float32, device=cuda_dev), out,
                 torch.tensor(d_np, dtype=torch.float32, device=cuda_dev), 0.5, 0.0, 1e-2, nonneg=False)
    torch.cuda.synchronize()
    ref = f_np - 0.5 * O.adjoint(og(g), O.forward(og(g), f_np) - d_np)
    assert rel(out.double().cpu().numpy() - f_np, ref - f_np) <= 2e-5

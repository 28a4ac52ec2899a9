"""Autograd wrappers, the DIP loop (Eq. (5)) and the TV loop (Eq. (4))."""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_19176_gb300 import Geometry, PatPlan, inputs
from paper_2604_19176_gb300.recon import (UNet, dip_reconstruct, operator_norm_sq, pat_apply, tv_reconstruct,
                                          tv_value)


def og(g):
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


# ---------------------------------------------------------------- CPU only

def test_unet_shapes_and_nonnegativity():
    net = UNet(in_ch=4, base=8)
    x = torch.randn(1, 4, 32, 32)
    y = net(x)
    assert y.shape == (1, 1, 32, 32)
    assert float(y.detach().min()) >= 0.0
    # encoder 8-16-32-64, decoder back to 8, head to 1
    assert net.enc[3][0].out_channels == 64 and net.dec[2][0].out_channels == 8
    m = UNet(in_ch=4, base=8, mouse=True)
    assert m.head.bias is None and m.head.kernel_size == (1, 1)
    # LeakyReLU(0.125) output: flipping the sign of the 1x1 head flips the sign
    # of every pre-activation, so the two outputs are y+ and -0.125 y+ apart
    with torch.no_grad():
        ya = m(x)
        m.head.weight.neg_()
        yb = m(x)
    pre = torch.where(ya >= 0, ya, ya / 0.125)        # undo the activation
    expect = torch.where(-pre >= 0, -pre, -0.125 * pre)
    assert torch.allclose(yb, expect, rtol=1e-5, atol=1e-6)
    assert float(torch.minimum(ya, yb).min()) < 0.0     # negative outputs occur


def test_unet_paper_channel_plan():
    net = UNet(in_ch=32, base=32)
    assert [b[0].out_channels for b in net.enc] == [32, 64, 128, 256]
    assert [u.out_channels for u in net.up] == [128, 64, 32]


# ---------------------------------------------------------------- GPU

@pytest.mark.gpu
def test_operator_autograd_matches_oracle_gradient(cuda_dev):
    """32x32 sub-problem: autograd through A gives 2 A^T (A f - g) (oracle, FP64)
    and matches central differences of the quadratic loss."""
    g = Geometry(32, 16, 0.3, 1.4 * math.pi, 48, 2.0, 64)
    plan = PatPlan(g, device=cuda_dev)
    f = torch.tensor(inputs.random_image(32, seed=1), dtype=torch.float32, device=cuda_dev, requires_grad=True)
    d = torch.tensor(inputs.random_data(16, 48, seed=2), dtype=torch.float32, device=cuda_dev)
    loss = ((pat_apply(f, plan) - d) ** 2).sum()
    loss.backward()
    fn = f.detach().double().cpu().numpy()
    ref = 2.0 * O.adjoint(og(g), O.forward(og(g), fn) - d.double().cpu().numpy())
    got = f.grad.double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    # directional finite difference (exact for a quadratic up to rounding)
    v = torch.tensor(inputs.random_image(32, seed=3), dtype=torch.float32, device=cuda_dev)
    with torch.no_grad():
        L = lambda x: float(((plan.forward(x).double() - d.double()) ** 2).sum())
        fd = (L(f + v) - L(f - v)) / 2.0
    dd = float((f.grad.double() * v.double()).sum())
    assert abs(fd - dd) <= 1e-4 * max(abs(dd), 1.0)


@pytest.mark.gpu
def test_tv_autograd_matches_oracle(cuda_dev):
    g = Geometry(32, 8, 0.0, math.pi, 16, 2.0, 16)
    plan = PatPlan([g, g], device=cuda_dev)
    imgs = np.stack([inputs.vessel_phantom(32, 4, seed=5), inputs.random_image(32, seed=6)]).astype(np.float32)
    f = torch.tensor(imgs, device=cuda_dev, requires_grad=True)
    w = torch.tensor([0.7, -1.3], device=cuda_dev)
    (tv_value(f, plan, 1e-2) * w).sum().backward()
    for i in range(2):
        _, rg = O.tv(imgs[i].astype(np.float64), 1e-2)
        got = f.grad[i].double().cpu().numpy()
        assert np.linalg.norm(got - float(w[i]) * rg) / np.linalg.norm(float(w[i]) * rg) <= 1e-5
    # directional central difference of the GPU TV value itself (FP32): smooth
    # images, eps = 0.1 and step 1e-2 keep the FP32 rounding of the difference
    # quotient near 3e-4 (measured on a CPU emulation of the same sums)
    sm = np.stack([inputs.gaussian_phantom(32, 3, seed=5), inputs.vessel_phantom(32, 4, seed=5)]).astype(np.float32)
    fs = torch.tensor(sm, device=cuda_dev, requires_grad=True)
    (tv_value(fs, plan, 0.1) * w).sum().backward()
    v = torch.tensor(inputs.gaussian_phantom(32, 4, seed=9), dtype=torch.float32, device=cuda_dev).expand(2, 32, 32)
    with torch.no_grad():
        t = 1e-2
        fd = ((tv_value(fs + t * v, plan, 0.1) - tv_value(fs - t * v, plan, 0.1)).double() / (2 * t)) @ w.double()
    dd = float((fs.grad.double() * v.double()).sum())
    assert abs(float(fd) - dd) <= 2e-3 * abs(dd)


@pytest.mark.gpu
def test_tv_reconstruction_decreases_objective(cuda_dev):
    g = Geometry(64, 64, 0.0, 2 * math.pi, 128, 2.0, 128)
    plan = PatPlan(g, device=cuda_dev)
    f_true = torch.tensor(inputs.gaussian_phantom(64, 5, seed=1), dtype=torch.float32, device=cuda_dev)
    data = plan.forward(f_true)
    alpha, eps = 1e-3, 1e-3
    objs = []

    def obj(k, f, r):
        if k % 10 == 0:
            res = plan.forward(f) - data
            objs.append(0.5 * float((res.double() ** 2).sum()) + alpha * float(plan.tv_value(f, eps)[0]))

    f, hist = tv_reconstruct(plan, data, alpha, eps=eps, iters=120, callback=obj)
    assert float(f.min()) >= 0.0
    assert all(b <= a * (1 + 1e-6) for a, b in zip(objs, objs[1:]))
    err0 = float(f_true.norm())
    assert float((f - f_true).norm()) < 0.5 * err0


@pytest.mark.gpu
def test_dip_loop_runs_and_resumes(cuda_dev, tmp_path):
    g = Geometry(32, 16, 0.0, 1.5 * math.pi, 48, 2.0, 64)
    plan = PatPlan(g, device=cuda_dev)
    f_true = torch.tensor(inputs.gaussian_phantom(32, 3, seed=2), dtype=torch.float32, device=cuda_dev)
    data = plan.forward(f_true)
    z = torch.tensor(inputs.dip_input(4, 32, seed=3), dtype=torch.float32, device=cuda_dev)
    net = UNet(in_ch=4, base=8).to(cuda_dev)
    f, hist, _ = dip_reconstruct(plan, data, z, lam=1e-4, steps=40, lr=1e-3, net=net, callback=lambda *a: None)
    assert hist[-1] < hist[0]
    assert f.shape == (32, 32) and float(f.min()) >= 0.0
    ck = str(tmp_path / "dip.pt")
    _, h1, _ = dip_reconstruct(plan, data, z, steps=6, lr=1e-3, net=UNet(in_ch=4, base=8).to(cuda_dev),
                               checkpoint=ck, checkpoint_every=3)
    assert os.path.exists(ck) and len(h1) == 6
    _, h2, _ = dip_reconstruct(plan, data, z, steps=9, lr=1e-3, net=UNet(in_ch=4, base=8).to(cuda_dev),
                               checkpoint=ck, checkpoint_every=3)
    assert len(h2) == 9 and h2[:6] == h1


@pytest.mark.gpu
def test_operator_norm_positive(cuda_dev):
    plan = PatPlan(Geometry(32, 16, 0.0, math.pi, 48, 2.0, 64), device=cuda_dev)
    assert operator_norm_sq(plan, iters=10) > 0

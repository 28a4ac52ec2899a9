"""Reconstruction loops on top of the operator library.

* :class:`PatOperator` — torch.autograd.Function: forward = A (``pat_forward``),
  backward = A^T (``pat_adjoint``), the adjoint the data term's gradient needs
  (Sec. 2.2).
* :class:`TVFunction` — smoothed TV with its hand-written gradient
  (``pat_tv_grad``) as the backward.
* :class:`UNet` — the DIP network of Sec. 2.2.1 in stock PyTorch: four encoder
  stages of two 3x3 conv + BN + ReLU (32, 64, 128, 256 channels) joined by 2x2
  max pooling, three decoder stages (transposed conv, skip concatenation, two
  3x3 conv + BN + ReLU), a final 3x3 conv to one channel and ReLU.
* :func:`dip_reconstruct` — Eq. (5): minimise ||A phi_theta(z) - g||^2 +
  lambda TV(phi_theta(z)) over the network parameters with Adam (optional
  cosine schedule, checkpoint / resume).
* :func:`tv_reconstruct` — Eq. (4): projected gradient descent on
  1/2 ||A f - g||^2 + alpha TV(f) with f >= 0, stopped by the relative-change
  rule of Sec. 2.3; every step runs in the library's kernels.
* :func:`pdhg_reconstruct` — Eq. (4) with the unsmoothed TV, solved by the
  primal-dual hybrid gradient method the paper uses (Sec. 2.1), one
  ``pat_pdhg_step`` per iteration, same stopping rule.
* :func:`initial_reconstruction` — an approximate inverse (A^T, Landweber or
  CGLS) as the DIP network input in place of random noise (Sec. 2.2).
"""
from __future__ import annotations

import math
import os
from typing import Callable, Optional

import torch
import torch.nn as nn
import torch.nn.functional as F

from .api import PatPlan

__all__ = ["PatOperator", "TVFunction", "UNet", "operator_norm_sq", "dip_reconstruct", "tv_reconstruct", "pat_apply",
           "tv_value", "pdhg_steps", "pdhg_reconstruct", "initial_reconstruction"]


class PatOperator(torch.autograd.Function):
    """g = A f with dL/df = A^T dL/dg (exact discrete adjoint)."""

    @staticmethod
    def forward(ctx, f: torch.Tensor, plan: PatPlan) -> torch.Tensor:
        ctx.plan = plan
        return plan.forward(f.contiguous())

    @staticmethod
    def backward(ctx, grad_g: torch.Tensor):
        return ctx.plan.adjoint(grad_g.contiguous()), None


class TVFunction(torch.autograd.Function):
    """Per-instance smoothed isotropic TV values; backward scales dTV/df."""

    @staticmethod
    def forward(ctx, f: torch.Tensor, plan: PatPlan, eps: float) -> torch.Tensor:
        val, grad = plan.tv_grad(f.contiguous(), eps)
        ctx.save_for_backward(grad)
        ctx.plan = plan
        return val

    @staticmethod
    def backward(ctx, grad_val: torch.Tensor):
        (grad,) = ctx.saved_tensors
        plan = ctx.plan
        if len(plan.geoms) == 1:
            return grad * grad_val.reshape(()), None, None
        if plan.uniform:
            return grad * grad_val.reshape(-1, 1, 1), None, None
        out = torch.empty_like(grad)
        for i, (a, b) in enumerate(zip(plan.f_offsets[:-1], plan.f_offsets[1:])):
            out[a:b] = grad[a:b] * grad_val[i]
        return out, None, None


def pat_apply(f: torch.Tensor, plan: PatPlan) -> torch.Tensor:
    return PatOperator.apply(f, plan)


def tv_value(f: torch.Tensor, plan: PatPlan, eps: float) -> torch.Tensor:
    return TVFunction.apply(f, plan, eps)


class _Block(nn.Sequential):
    def __init__(self, cin: int, cout: int):
        super().__init__(
            nn.Conv2d(cin, cout, 3, padding=1), nn.BatchNorm2d(cout), nn.ReLU(inplace=True),
            nn.Conv2d(cout, cout, 3, padding=1), nn.BatchNorm2d(cout), nn.ReLU(inplace=True))


class UNet(nn.Module):
    """Four-level U-Net of Sec. 2.2.1 (``mouse=True``: 1x1 bias-free head and
    LeakyReLU(0.125) output instead of 3x3 conv + ReLU)."""

    def __init__(self, in_ch: int = 32, base: int = 32, out_ch: int = 1, mouse: bool = False):
        super().__init__()
        c = [base, 2 * base, 4 * base, 8 * base]
        self.enc = nn.ModuleList([_Block(in_ch, c[0]), _Block(c[0], c[1]), _Block(c[1], c[2]), _Block(c[2], c[3])])
        self.up = nn.ModuleList([nn.ConvTranspose2d(c[3], c[2], 2, stride=2), nn.ConvTranspose2d(c[2], c[1], 2, stride=2),
                                 nn.ConvTranspose2d(c[1], c[0], 2, stride=2)])
        self.dec = nn.ModuleList([_Block(2 * c[2], c[2]), _Block(2 * c[1], c[1]), _Block(2 * c[0], c[0])])
        self.head = nn.Conv2d(c[0], out_ch, 1, bias=False) if mouse else nn.Conv2d(c[0], out_ch, 3, padding=1)
        self.mouse = mouse

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        skips = []
        for i, blk in enumerate(self.enc):
            x = blk(x)
            if i < 3:
                skips.append(x)
                x = F.max_pool2d(x, 2)
        for up, dec in zip(self.up, self.dec):
            x = up(x)
            x = dec(torch.cat([x, skips.pop()], dim=1))
        x = self.head(x)
        return F.leaky_relu(x, 0.125) if self.mouse else F.relu(x)


@torch.no_grad()
def operator_norm_sq(plan: PatPlan, iters: int = 30, seed: int = 0) -> float:
    """||A||^2 by power iteration on A^T A."""
    gen = torch.Generator(device=plan.device).manual_seed(seed)
    x = torch.rand(plan.image_shape(), generator=gen, device=plan.device, dtype=torch.float32)
    lam = 0.0
    for _ in range(iters):
        y = plan.adjoint(plan.forward(x))
        lam = float(y.norm())
        x = y / max(lam, 1e-30)
    return lam


@torch.no_grad()
def tv_reconstruct(plan: PatPlan, g: torch.Tensor, alpha: float, eps: float = 1e-3, iters: int = 500,
                   tau: Optional[float] = None, nonneg: bool = True, stop_tol: float = 1e-4,
                   f0: Optional[torch.Tensor] = None, callback: Optional[Callable] = None) -> tuple:
    """Projected gradient descent for Eq. (4): min_{f >= 0} 1/2 ||A f - g||^2 + alpha TV_eps(f).

    Step tau = 1 / (||A||^2 + 8 alpha / eps) (a Lipschitz bound of the
    gradient).  Stops when ||f_k - f_{k-1}|| / ||f_k|| <= stop_tol for every
    instance (Sec. 2.3).  Returns (f, history of relative changes).
    """
    if tau is None:
        tau = 1.0 / (operator_norm_sq(plan) + 8.0 * alpha / eps)
    f = torch.zeros(plan.image_shape(), dtype=torch.float32, device=plan.device) if f0 is None else f0.clone()
    gp = torch.empty(plan.data_shape(), dtype=torch.float32, device=plan.device)
    adj = torch.empty_like(f)
    tvg = torch.empty_like(f)
    delta = torch.empty(2 * len(plan.geoms), dtype=torch.float32, device=plan.device)
    hist = []
    for k in range(iters):
        plan.forward(f, out=gp)
        plan.residual(gp, g, out=gp)
        plan.adjoint(gp, out=adj)
        plan.tv_grad(f, eps, grad=tvg, want_value=False)
        plan.descent_step(f, adj, tvg, tau, alpha, nonneg=nonneg, delta=delta)
        d = delta.view(-1, 2)
        rel = torch.sqrt(d[:, 0] / torch.clamp(d[:, 1], min=1e-30))
        r = float(rel.max())
        hist.append(r)
        if callback is not None:
            callback(k, f, r)
        if k > 0 and r <= stop_tol:
            break
    return f, hist


def pdhg_steps(plan: PatPlan, beta: float = 0.0) -> tuple:
    """Step sizes (sigma, tau) for the primal-dual iteration: sigma = tau =
    0.99 / ||K|| with ||K||^2 <= ||A||^2 + 8 (||grad||^2 <= 8 for forward
    differences).  With the mean penalty (beta > 0, gradient Lipschitz constant
    beta / P) tau is lowered until 1/tau - sigma ||K||^2 >= beta / (2 P), with
    sigma tau ||K||^2 = 0.98 kept."""
    k2 = operator_norm_sq(plan) + 8.0
    tau = 0.99 / math.sqrt(k2)
    if beta > 0:
        p_min = min(g.n * g.n for g in plan.geoms)
        tau = min(tau, 0.02 * 2.0 * p_min / beta)
    return 0.98 / (tau * k2), tau


@torch.no_grad()
def pdhg_reconstruct(plan: PatPlan, g: torch.Tensor, alpha: float, iters: int = 1000,
                     sigma: Optional[float] = None, tau: Optional[float] = None, nonneg: bool = True,
                     mean_penalty: Optional[tuple] = None, stop_tol: float = 1e-4, check_every: int = 1,
                     state: Optional[dict] = None, callback: Optional[Callable] = None) -> tuple:
    """Primal-dual hybrid gradient (Chambolle-Pock) for Eq. (4):
    min_{f >= 0} 1/2 ||A f - g||^2 + alpha TV(f), the paper's TV baseline
    solver (Sec. 2.1); each iteration is one ``pat_pdhg_step``.

    The mouse-data variant (Sec. 2.1) is ``nonneg=False`` with
    ``mean_penalty=(beta, c)``: + beta/2 (mean(f) - c)^2 per instance.
    Stops when ||f_k - f_{k-1}|| / ||f_k|| <= stop_tol for every instance
    (Sec. 2.3), tested every ``check_every`` iterations (the test reads two
    numbers per instance back to the host).  ``state`` (f, fbar, y, px, py,
    and fmean with the penalty) resumes a run.  Returns (f, history of
    (iteration, max relative change), state).
    """
    beta, c = mean_penalty if mean_penalty is not None else (0.0, 0.0)
    if sigma is None or tau is None:
        s0, t0 = pdhg_steps(plan, beta)
        sigma = s0 if sigma is None else sigma
        tau = t0 if tau is None else tau
    dev = plan.device
    if state is None:
        z = lambda shape: torch.zeros(shape, dtype=torch.float32, device=dev)  # noqa: E731
        state = {"f": z(plan.image_shape()), "fbar": z(plan.image_shape()), "y": z(plan.data_shape()),
                 "px": z(plan.image_shape()), "py": z(plan.image_shape())}
    if beta > 0 and "fmean" not in state:
        fo = plan.layout()[0]
        flat = state["f"].reshape(-1)
        state["fmean"] = torch.stack([flat[fo[i]:fo[i + 1]].mean() for i in range(len(plan.geoms))]).float()
    delta = torch.empty(2 * len(plan.geoms), dtype=torch.float32, device=dev)
    hist = []
    for k in range(iters):
        check = (k + 1) % check_every == 0 or k + 1 == iters
        plan.pdhg_step(state["f"], state["fbar"], state["y"], state["px"], state["py"], g, sigma, tau, alpha,
                       nonneg=nonneg, delta=delta if check else None, beta=beta, mean_target=c,
                       fmean=state.get("fmean") if beta > 0 else None)
        if check:
            d = delta.view(-1, 2)
            r = float(torch.sqrt(d[:, 0] / torch.clamp(d[:, 1], min=1e-30)).max())
            hist.append((k, r))
            if callback is not None:
                callback(k, state["f"], r)
            if k > 0 and r <= stop_tol:
                break
    return state["f"], hist, state


class _Segments:
    """Per-instance reductions and broadcasts over a plan's packed images / data."""

    def __init__(self, plan: PatPlan):
        dev = plan.device
        fo, go = plan.layout()
        n = len(plan.geoms)
        self.n = n
        self.f_idx = torch.repeat_interleave(torch.arange(n, device=dev),
                                             torch.tensor([fo[i + 1] - fo[i] for i in range(n)], device=dev))
        self.g_idx = torch.repeat_interleave(torch.arange(n, device=dev),
                                             torch.tensor([go[i + 1] - go[i] for i in range(n)], device=dev))

    def dot(self, a: torch.Tensor, b: torch.Tensor, image: bool) -> torch.Tensor:
        idx = self.f_idx if image else self.g_idx
        out = torch.zeros(self.n, dtype=torch.float64, device=a.device)
        return out.index_add_(0, idx, (a.reshape(-1).double() * b.reshape(-1).double()))

    def expand(self, v: torch.Tensor, image: bool, like: torch.Tensor) -> torch.Tensor:
        idx = self.f_idx if image else self.g_idx
        return v.float()[idx].reshape(like.shape)


@torch.no_grad()
def initial_reconstruction(plan: PatPlan, g: torch.Tensor, method: str = "cgls", iters: int = 10,
                           omega: Optional[float] = None) -> torch.Tensor:
    """Approximate inverse z ~ A^{-1} g for the DIP input (Sec. 2.2), standing in
    for the paper's fast FFT-based inverse, which is not described there.

    ``adjoint``: z = A^T g / ||A||^2.  ``landweber``: ``iters`` steps
    f <- f + omega A^T (g - A f) from 0 (omega = 1 / ||A||^2 by default).
    ``cgls``: ``iters`` conjugate-gradient steps on the normal equations from
    0, with step lengths per instance.  A and A^T are the library's kernels;
    the vector updates are plain tensor arithmetic, with FP64 inner products.
    """
    if method == "adjoint":
        return plan.adjoint(g) / operator_norm_sq(plan)
    if method == "landweber":
        w = 1.0 / operator_norm_sq(plan) if omega is None else omega
        f = torch.zeros(plan.image_shape(), dtype=torch.float32, device=plan.device)
        for _ in range(iters):
            f += w * plan.adjoint(g - plan.forward(f))
        return f
    if method != "cgls":
        raise ValueError(f"unknown method {method!r}")
    seg = _Segments(plan)
    f = torch.zeros(plan.image_shape(), dtype=torch.float32, device=plan.device)
    r = g.clone()
    s = plan.adjoint(r)
    p = s.clone()
    gamma = seg.dot(s, s, True)
    for _ in range(iters):
        q = plan.forward(p)
        qq = seg.dot(q, q, False)
        a = torch.where(qq > 0, gamma / torch.where(qq > 0, qq, 1.0), 0.0)
        f += seg.expand(a, True, f) * p
        r -= seg.expand(a, False, r) * q
        s = plan.adjoint(r)
        gamma_new = seg.dot(s, s, True)
        b = torch.where(gamma > 0, gamma_new / torch.where(gamma > 0, gamma, 1.0), 0.0)
        p = s + seg.expand(b, True, p) * p
        gamma = gamma_new
    return f


def dip_reconstruct(plan: PatPlan, g: torch.Tensor, z: torch.Tensor, lam: float = 1e-4, eps: float = 1e-3,
                    steps: int = 2000, lr: float = 1e-4, cosine: bool = False, net: Optional[nn.Module] = None,
                    checkpoint: Optional[str] = None, checkpoint_every: int = 100,
                    callback: Optional[Callable] = None, seed: int = 0,
                    mean_penalty: Optional[tuple] = None) -> tuple:
    """DIP of Eq. (5): theta* = argmin ||A phi_theta(z) - g||^2 + lam TV(phi_theta(z)).

    Adam at ``lr`` (cosine annealing over all steps if ``cosine``).  With
    ``checkpoint`` set, network/optimiser state and the step counter are saved
    every ``checkpoint_every`` steps and resumed from if the file exists.
    ``mean_penalty=(beta, c)`` adds beta (mean(f) - c)^2, the mean-intensity
    term of the mouse-data variant (Sec. 2.2; use with ``UNet(mouse=True)``).
    Returns (f = phi_theta(z), loss history).
    """
    dev = plan.device
    if net is None:
        torch.manual_seed(seed)
        net = UNet(in_ch=z.shape[1]).to(dev)
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=steps) if cosine else None
    start = 0
    hist: list = []
    if checkpoint and os.path.exists(checkpoint):
        st = torch.load(checkpoint, map_location=dev)
        net.load_state_dict(st["net"])
        opt.load_state_dict(st["opt"])
        if sched is not None and st.get("sched") is not None:
            sched.load_state_dict(st["sched"])
        start, hist = st["step"], st["hist"]
    img_shape = plan.image_shape()
    for k in range(start, steps):
        opt.zero_grad(set_to_none=True)
        f = net(z).reshape(img_shape)
        r = pat_apply(f, plan) - g
        loss = (r * r).sum() + lam * tv_value(f, plan, eps).sum()
        if mean_penalty is not None:
            loss = loss + mean_penalty[0] * (f.mean() - mean_penalty[1]) ** 2
        loss.backward()
        opt.step()
        if sched is not None:
            sched.step()
        hist.append(float(loss.detach()) if callback is not None or checkpoint else math.nan)
        if callback is not None:
            callback(k, f, hist[-1])
        if checkpoint and ((k + 1) % checkpoint_every == 0 or k + 1 == steps):
            torch.save({"net": net.state_dict(), "opt": opt.state_dict(),
                        "sched": sched.state_dict() if sched is not None else None, "step": k + 1, "hist": hist},
                       checkpoint + ".tmp")
            os.replace(checkpoint + ".tmp", checkpoint)
    with torch.no_grad():
        f = net(z).reshape(img_shape)
    return f, hist, net

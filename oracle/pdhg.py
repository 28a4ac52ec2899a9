"""FP64 primal-dual hybrid gradient (Chambolle-Pock) TV reconstruction.

Test infrastructure only: the product library neither imports nor links this
module.  It solves the TV-regularised problem of Eq. (4),

    min_{f >= 0}  1/2 ||A f - g||^2 + alpha TV(f),

with the primal-dual hybrid gradient method the paper uses for its TV
baseline (Sec. 2.1), and reports the relative change between consecutive
iterates that the paper's stopping rule tests (Sec. 2.3: converged when
||f_k - f_{k-1}|| / ||f_k|| <= 1e-4).

TV(f) is the unsmoothed isotropic total variation sum_i |(grad f)_i| with the
forward differences of ``tv`` in ``pat_oracle.c`` (zero difference on the last
column / row).  The problem is written as min_f F(K f) + G(f) with
K f = (A f, grad f), F(z, q) = 1/2 ||z - g||^2 + alpha sum_i |q_i| and
G = indicator of f >= 0 (or 0 when ``nonneg`` is false), and every iteration
takes the method's steps in order:

    y    <- prox_{sigma F1*}(y + sigma A fbar)       = (y + sigma (A fbar - g)) / (1 + sigma)
    p    <- prox_{sigma F2*}(p + sigma grad fbar)    = projection of each p_i onto |p_i| <= alpha
    f'   <- prox_{tau G}(f - tau (A^T y + grad^T p)) = max(f - tau (...), 0)
    fbar <- 2 f' - f                                 (extrapolation, theta = 1)

The operator A and its adjoint are passed in (the FP64 oracle, or a dense
matrix in the pins), so the iteration is checked independently of them.

For the experimental mouse data the paper drops f >= 0 and adds a quadratic
penalty on the mean intensity (Sec. 2.1, Sec. 2.2).  With ``mean_penalty =
(beta, c)`` the objective gains h(f) = beta/2 (mean(f) - c)^2.  h is smooth with
gradient beta (mean(f) - c) / P on every pixel (P pixels) and Lipschitz constant
beta / P, so it enters the primal step as an explicit gradient term (the
primal-dual method with a smooth term, Condat 2013 / Vu 2013):

    f' <- prox_{tau G}(f - tau (A^T y + grad^T p + grad h(f)))

which converges when 1/tau - sigma ||K||^2 >= beta / (2 P).
"""
from __future__ import annotations

import numpy as np

__all__ = ["grad", "grad_adjoint", "pdhg"]


def grad(f: np.ndarray):
    """Forward differences (gx, gy) of an N x N image; 0 on the last column / row."""
    gx = np.zeros_like(f)
    gy = np.zeros_like(f)
    gx[:, :-1] = f[:, 1:] - f[:, :-1]
    gy[:-1, :] = f[1:, :] - f[:-1, :]
    return gx, gy


def grad_adjoint(px: np.ndarray, py: np.ndarray) -> np.ndarray:
    """grad^T (px, py): the exact adjoint of ``grad`` (minus the divergence)."""
    out = np.zeros_like(px)
    out[:, :-1] -= px[:, :-1]
    out[:, 1:] += px[:, :-1]
    out[:-1, :] -= py[:-1, :]
    out[1:, :] += py[:-1, :]
    return out


def pdhg(A, At, g: np.ndarray, n: int, alpha: float, sigma: float, tau: float, iters: int, nonneg: bool = True,
         state=None, mean_penalty=None):
    """Run ``iters`` iterations; returns (state, relative changes per iteration).

    A(f) maps an n x n image to data shaped like g; At is its adjoint.  state is
    a dict with f, fbar, y, px, py (zeros when None), updated copies returned.
    mean_penalty = (beta, c) adds beta/2 (mean(f) - c)^2 to the objective.
    """
    if state is None:
        z = np.zeros((n, n))
        state = {"f": z.copy(), "fbar": z.copy(), "y": np.zeros_like(g, dtype=np.float64), "px": z.copy(),
                 "py": z.copy()}
    f, fbar, y = state["f"].copy(), state["fbar"].copy(), state["y"].copy()
    px, py = state["px"].copy(), state["py"].copy()
    rel = []
    for _ in range(iters):
        y = (y + sigma * (A(fbar) - g)) / (1.0 + sigma)
        gx, gy = grad(fbar)
        qx, qy = px + sigma * gx, py + sigma * gy
        scale = np.maximum(1.0, np.sqrt(qx * qx + qy * qy) / alpha) if alpha > 0 else None
        px, py = (qx / scale, qy / scale) if alpha > 0 else (np.zeros_like(qx), np.zeros_like(qy))
        step = At(y) + grad_adjoint(px, py)
        if mean_penalty is not None:
            beta, c = mean_penalty
            step = step + beta * (f.mean() - c) / f.size
        f_new = f - tau * step
        if nonneg:
            f_new = np.maximum(f_new, 0.0)
        fbar = 2.0 * f_new - f
        nrm = np.linalg.norm(f_new)
        rel.append(np.linalg.norm(f_new - f) / nrm if nrm > 0 else 0.0)
        f = f_new
    return {"f": f, "fbar": fbar, "y": y, "px": px, "py": py}, rel

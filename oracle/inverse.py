"""FP64 approximate inverses of A for the DIP input (test infrastructure only).

The paper feeds the network an initial reconstruction z = A^{-1} g from a
fast FFT-based inverse of its prior work (Sec. 2.2), which it does not
describe.  The stand-ins here are the classical regularising iterations on
the normal equations A^T A f = A^T g, started from f = 0:

* Landweber:  f <- f + omega A^T (g - A f),  0 < omega < 2 / ||A||^2;
* CGLS (conjugate gradients on the normal equations, Hestenes-Stiefel form
  for least squares): after k steps f_k minimises ||A f - g|| over the Krylov
  space span{A^T g, (A^T A) A^T g, ..., (A^T A)^{k-1} A^T g}.

The product library neither imports nor links this module.  A and A^T are
passed in as callables.
"""
from __future__ import annotations

import numpy as np

__all__ = ["landweber", "cgls"]


def landweber(A, At, g: np.ndarray, shape, omega: float, iters: int) -> np.ndarray:
    f = np.zeros(shape)
    for _ in range(iters):
        f = f + omega * At(g - A(f))
    return f


def cgls(A, At, g: np.ndarray, shape, iters: int):
    """Returns (f_k, residual norms ||g - A f_i|| for i = 0..k)."""
    f = np.zeros(shape)
    r = np.array(g, dtype=np.float64)          # g - A f
    s = At(r)                                  # A^T r, the normal-equation residual
    p = s.copy()
    gamma = float(np.sum(s * s))
    res = [float(np.linalg.norm(r))]
    for _ in range(iters):
        if gamma == 0.0:
            break
        q = A(p)
        a = gamma / float(np.sum(q * q))
        f = f + a * p
        r = r - a * q
        s = At(r)
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        res.append(float(np.linalg.norm(r)))
    return f, res

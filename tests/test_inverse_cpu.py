"""Pins of the FP64 approximate inverses (DIP input) against what linear
algebra fixes: the CGLS iterate is the least-squares minimiser over its Krylov
space (solved independently by an orthonormal basis and lstsq) and reaches
the full least-squares solution after n steps; Landweber's k-th iterate is
the spectral filter sum_{i<k} omega (I - omega A^T A)^i A^T g, evaluated
through the SVD."""
import math

import numpy as np

from oracle import inverse as I


def _problem(m, n, seed, cond=30.0):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.geomspace(1.0, 1.0 / cond, n)
    A = U @ np.diag(s) @ V.T
    g = rng.standard_normal(m)
    return A, g


def test_cgls_is_krylov_least_squares():
    A, g = _problem(30, 12, seed=1)
    for k in (1, 3, 6):
        f, res = I.cgls(lambda x: A @ x, lambda y: A.T @ y, g, (12,), k)
        # orthonormal basis of span{(A^T A)^i A^T g, i < k}
        B = [A.T @ g]
        for _ in range(k - 1):
            B.append(A.T @ (A @ B[-1]))
        Q, _ = np.linalg.qr(np.stack(B, axis=1))
        c = np.linalg.lstsq(A @ Q, g, rcond=None)[0]
        ref = Q @ c
        assert np.max(np.abs(f - ref)) < 1e-9 * np.max(np.abs(ref))
        assert all(res[i + 1] <= res[i] + 1e-12 for i in range(len(res) - 1))


def test_cgls_reaches_least_squares_in_n_steps():
    A, g = _problem(30, 8, seed=2, cond=5.0)
    f, _ = I.cgls(lambda x: A @ x, lambda y: A.T @ y, g, (8,), 8)
    ref = np.linalg.lstsq(A, g, rcond=None)[0]
    assert np.max(np.abs(f - ref)) < 1e-9


def test_landweber_spectral_filter():
    A, g = _problem(25, 10, seed=3)
    omega = 1.0 / np.linalg.norm(A, 2) ** 2
    k = 7
    f = I.landweber(lambda x: A @ x, lambda y: A.T @ y, g, (10,), omega, k)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    filt = (1.0 - (1.0 - omega * s * s) ** k) / s      # sum_{i<k} omega (1 - omega s^2)^i s
    ref = Vt.T @ (filt * (U.T @ g))
    assert np.max(np.abs(f - ref)) < 1e-12 * math.sqrt(len(g))

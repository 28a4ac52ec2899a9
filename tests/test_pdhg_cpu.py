"""Pins of the FP64 primal-dual (Chambolle-Pock) TV solver of Eq. (4).

The solver takes A and A^T as callables, so these pins drive it with small
dense matrices and check its result against what the problem itself fixes:
the non-negative least-squares solution for alpha = 0 (scipy's NNLS), the
constant-image solution once alpha is large, and the optimality conditions of
Eq. (4) for 0 < alpha.  The difference operator is pinned against the C
oracle's TV and against an explicit matrix built from unit vectors.
"""
import math

import numpy as np
import pytest
from scipy import optimize

from oracle import pdhg as P
from paper_2604_19176_gb300 import inputs


def _diff_matrix(n):
    """The forward-difference operator as an explicit (2 n^2) x n^2 matrix."""
    D = np.zeros((2 * n * n, n * n))
    for i in range(n):
        for j in range(n):
            r = i * n + j
            if j + 1 < n:
                D[r, r + 1], D[r, r] = 1.0, -1.0
            if i + 1 < n:
                D[n * n + r, r + n], D[n * n + r, r] = 1.0, -1.0
    return D


def test_grad_matches_explicit_matrix_and_its_transpose():
    n = 7
    D = _diff_matrix(n)
    f = inputs.random_image(n, seed=4)
    gx, gy = P.grad(f)
    assert np.array_equal(np.concatenate([gx.ravel(), gy.ravel()]), D @ f.ravel())
    p = np.random.default_rng(5).standard_normal(2 * n * n)
    px, py = p[:n * n].reshape(n, n), p[n * n:].reshape(n, n)
    # rows with no difference (last column / row) carry no weight in D^T
    assert np.allclose(P.grad_adjoint(px, py).ravel(), D.T @ p, atol=1e-14, rtol=0)


def test_grad_agrees_with_c_oracle_tv(orc):
    """sum |grad f| is the C oracle's TV at eps = 0, and grad^T(grad f / s) is
    the gradient of its smoothed TV: two independent codes of the same operator."""
    n = 11
    f = inputs.random_image(n, seed=6)
    gx, gy = P.grad(f)
    assert abs(np.sum(np.hypot(gx, gy)) - orc.tv(f, 0.0, with_grad=False)) < 1e-12 * n * n
    eps = 0.05
    s = np.sqrt(gx * gx + gy * gy + eps * eps)
    _, g = orc.tv(f, eps)
    assert np.allclose(P.grad_adjoint(gx / s, gy / s), g, atol=1e-13, rtol=0)


def _problem(n, m, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n * n)) / math.sqrt(m)
    f0 = np.maximum(rng.standard_normal((n, n)), 0.0)
    g = A @ f0.ravel() + 0.3 * rng.standard_normal(m)
    return A, g


def _run(A, g, n, alpha, iters, nonneg=True, mean_penalty=None, tau=None):
    L = math.sqrt(np.linalg.norm(A, 2) ** 2 + 8.0)
    tau = 0.99 / L if tau is None else tau
    sigma = 0.98 / (tau * L * L)
    st, rel = P.pdhg(lambda f: A @ f.ravel(), lambda y: (A.T @ y).reshape(n, n), g, n, alpha, sigma, tau,
                     iters, nonneg=nonneg, mean_penalty=mean_penalty)
    return st, rel


def test_alpha_zero_is_nonnegative_least_squares():
    n = 4
    A, g = _problem(n, 40, seed=7)
    st, rel = _run(A, g, n, 0.0, 6000)
    ref, _ = optimize.nnls(A, g)
    assert np.any(ref == 0.0)   # the constraint is active somewhere
    assert np.max(np.abs(st["f"].ravel() - ref)) < 1e-8
    assert rel[-1] < 1e-9


def test_alpha_zero_without_constraint_is_least_squares():
    n = 4
    A, g = _problem(n, 40, seed=8)
    st, _ = _run(A, g, n, 0.0, 6000, nonneg=False)
    ref = np.linalg.lstsq(A, g, rcond=None)[0]
    assert np.max(np.abs(st["f"].ravel() - ref)) < 1e-8


@pytest.mark.parametrize("beta,c,tau", [(3.0, 0.4, None), (100.0, -0.2, 0.006)])
def test_mean_penalty_is_augmented_least_squares(beta, c, tau):
    """alpha = 0, no constraint, penalty beta/2 (mean f - c)^2: the minimiser is
    the least-squares solution of [A; sqrt(beta) 1^T / P] f = [g; sqrt(beta) c].
    The larger beta needs the smaller tau: 1/tau - sigma ||K||^2 >= beta / (2 P)."""
    n = 4
    A, g = _problem(n, 40, seed=12)
    P_ = n * n
    Aa = np.vstack([A, math.sqrt(beta) * np.ones((1, P_)) / P_])
    ref = np.linalg.lstsq(Aa, np.concatenate([g, [math.sqrt(beta) * c]]), rcond=None)[0]
    st, _ = _run(A, g, n, 0.0, 20000, nonneg=False, mean_penalty=(beta, c), tau=tau)
    assert np.max(np.abs(st["f"].ravel() - ref)) < 1e-8
    # the penalty moved the mean towards c
    free = np.linalg.lstsq(A, g, rcond=None)[0]
    assert abs(ref.mean() - c) < abs(free.mean() - c)


def test_large_alpha_gives_best_constant_image():
    """For alpha far above the data gradient's size the minimiser is the best
    constant c >= 0: c = max(0, <A 1, g> / ||A 1||^2)."""
    n = 4
    A, g = _problem(n, 40, seed=9)
    a1 = A @ np.ones(n * n)
    c = max(0.0, float(a1 @ g) / float(a1 @ a1))
    assert c > 0
    st, _ = _run(A, g, n, 1e3, 20000)
    assert np.max(np.abs(st["f"] - c)) < 1e-6


@pytest.mark.parametrize("alpha,has_zeros", [(0.05, True), (0.3, False)])
def test_optimality_conditions_for_tv(alpha, has_zeros):
    """At the solution of Eq. (4): y = A f - g; p_i = alpha grad f_i / |grad f_i|
    where grad f_i != 0 and |p_i| <= alpha elsewhere; w = A^T y + grad^T p is 0 on
    the support of f and >= 0 where f = 0.  The objective is also no larger than
    at random feasible perturbations."""
    n = 4
    A, g = _problem(n, 40, seed=10)
    st, rel = _run(A, g, n, alpha, 40000)
    f, y, px, py = st["f"], st["y"], st["px"], st["py"]
    assert rel[-1] < 1e-10
    assert np.max(np.abs(y - (A @ f.ravel() - g))) < 1e-7
    gx, gy = P.grad(f)
    mag = np.hypot(gx, gy)
    pm = np.hypot(px, py)
    assert np.all(pm <= alpha * (1 + 1e-12))
    on = mag > 1e-6
    assert on.any() and (~on).any()   # both kinds of pixel occur
    assert np.max(np.abs(px[on] - alpha * gx[on] / mag[on])) < 1e-5
    assert np.max(np.abs(py[on] - alpha * gy[on] / mag[on])) < 1e-5
    w = (A.T @ y).reshape(n, n) + P.grad_adjoint(px, py)
    supp = f > 1e-8
    assert supp.any() and (~supp).any() == has_zeros
    assert np.max(np.abs(w[supp])) < 1e-6
    if has_zeros:
        assert np.min(w[~supp]) > -1e-6

    def obj(x):
        x = x.reshape(n, n)
        ax, ay = P.grad(x)
        return 0.5 * np.sum((A @ x.ravel() - g) ** 2) + alpha * np.sum(np.hypot(ax, ay))

    best = obj(f)
    rng = np.random.default_rng(11)
    for _ in range(200):
        x = np.maximum(f + 1e-3 * rng.standard_normal((n, n)), 0.0)
        assert obj(x) >= best - 1e-12


def test_oracle_operator_run_decreases_relative_change(orc):
    """A short run on the discrete PAT operator: iterates stay non-negative and
    the relative change of consecutive iterates falls."""
    g_ = orc.Geometry(16, 12, 0.0, 1.5 * math.pi, 24, 2.0, 24)
    f0 = inputs.vessel_phantom(16, seed=3)
    g = orc.forward(g_, f0)
    A = np.zeros((g.size, 256))
    for i in range(256):
        e = np.zeros(256)
        e[i] = 1.0
        A[:, i] = orc.forward(g_, e.reshape(16, 16)).ravel()
    # the oracle's adjoint is the transpose of its forward
    d = inputs.random_data(12, 24, seed=4)
    assert np.allclose(orc.adjoint(g_, d).ravel(), A.T @ d.ravel(), atol=1e-12, rtol=0)
    L = math.sqrt(np.linalg.norm(A, 2) ** 2 + 8.0)
    st, rel = P.pdhg(lambda f: orc.forward(g_, f), lambda y: orc.adjoint(g_, y), g, 16, 1e-3, 0.99 / L, 0.99 / L, 300)
    assert np.all(st["f"] >= 0)
    assert rel[-1] < 0.1 * rel[5]

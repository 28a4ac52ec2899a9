"""Pins of the FP64 oracle against facts fixed by the mathematics and the paper.

Each test checks the oracle against something other than itself: closed
forms of the 2D wave problem (Eq. (1)-(3)), exact invariants of the discrete
operators, independent quadrature (QUADPACK) and brute force on tiny grids,
and the detector numbers the paper prints (Sec. 2.1, Sec. 2.4.2).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from paper_2604_19176_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def geom(orc, n, n_det, n_t, K, span=2 * math.pi, start=0.0, t_max=2.0):
    return orc.Geometry(n, n_det, start, span, n_t, t_max, K)


# --------------------------------------------------------------------------
# Abel integral + midpoint derivative
# --------------------------------------------------------------------------

@pytest.mark.parametrize("tau", [0.5, 1.5, 2.5, 10.5, 77.5, 511.5, 2048.5])
def test_abel_weight_moments(orc, tau):
    """Hats reproduce 1 and rho, so sum_m w_m = int_0^tau rho/S = tau and
    sum_m m w_m = int_0^tau rho^2/S = pi tau^2 / 4 exactly."""
    n_r = int(math.ceil(tau)) + 2
    w = orc.abel_weights(tau, n_r)
    m = np.arange(n_r)
    assert abs(w.sum() - tau) / tau < 1e-13
    assert abs(w @ m - math.pi * tau * tau / 4) / (math.pi * tau * tau / 4) < 1e-13
    assert np.all(w[int(math.ceil(tau)) + 1:] == 0)


@pytest.mark.parametrize("n_t", [8, 128, 512, 2048])
def test_abel_matrix_invariants(orc, n_t):
    """P.1 = 1 (Q(t) = t for M = 1) and P.r = pi t / 2 (Q = pi t^2/4 for M = r,
    exact under the midpoint difference).  P row k is a difference of weight
    vectors of size ~k, so the absolute error allowance grows with k."""
    P = orc.abel_matrix(n_t)
    k = np.arange(1, n_t + 1)
    assert np.all(np.abs(P @ np.ones(n_t + 2) - 1.0) <= 1e-13 * (k + 1) + 1e-14)
    assert np.all(np.abs(P @ np.arange(n_t + 2) - math.pi * k / 2) <= 1e-13 * (k + 1) ** 2)
    # lower-triangular with one extra super-diagonal: P[k-1, m] = 0 for m > k + 1
    for kk in range(n_t):
        assert np.all(P[kk, kk + 3:] == 0.0)


def _w_quad(tau, m):
    """w_m(tau) by QUADPACK; the endpoint singularity (tau - rho)^(-1/2) is
    handled by the algebraic weight of qawse."""
    total = 0.0
    for a, b, hat in ((m - 1, m, lambda r: r - (m - 1)), (m, m + 1, lambda r: (m + 1) - r)):
        a = max(a, 0.0)
        b = min(b, tau)
        if a >= b:
            continue
        if b >= tau:  # singular endpoint at rho = tau
            f = lambda r, hat=hat: hat(r) * r / math.sqrt(tau + r)
            total += integrate.quad(f, a, b, weight="alg", wvar=(0.0, -0.5), epsabs=1e-15, epsrel=1e-14)[0]
        else:
            f = lambda r, hat=hat: hat(r) * r / math.sqrt((tau - r) * (tau + r))
            total += integrate.quad(f, a, b, epsabs=1e-15, epsrel=1e-14)[0]
    return total


@pytest.mark.parametrize("tau,m", [(0.5, 0), (0.5, 1), (1.5, 0), (1.5, 2), (3.5, 1), (3.5, 4), (40.5, 0),
                                   (40.5, 17), (40.5, 40), (40.5, 41), (300.5, 299), (300.5, 3)])
def test_abel_weights_vs_quadpack(orc, tau, m):
    w = orc.abel_weights(tau, int(math.ceil(tau)) + 2)
    ref = _w_quad(tau, m)
    assert abs(w[m] - ref) <= 1e-11 * max(abs(ref), 1e-3)


def test_abel_dawson_closed_form(orc):
    """A Gaussian centred on the detector has circular means exp(-r^2/s^2), and
    p(t) = d/dt int_0^t r e^{-r^2/s^2} / sqrt(t^2 - r^2) dr = 1 - 2 (t/s) D(t/s)
    (D = Dawson's integral).  The product-integrated Abel stage must converge
    to it at second order in Delta."""
    s, T = 0.1, 2.0
    errs = []
    for n_t in (128, 256, 512, 1024):
        P = orc.abel_matrix(n_t)
        d = T / n_t
        r = np.arange(n_t + 2) * d
        t = np.arange(1, n_t + 1) * d
        p = 1.0 - 2.0 * (t / s) * special.dawsn(t / s)
        errs.append(np.linalg.norm(P @ np.exp(-(r / s) ** 2) - p) / np.linalg.norm(p))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.6 < q < 4.4 for q in ratios), (errs, ratios)
    assert errs[-1] < 2e-4


# --------------------------------------------------------------------------
# Bilinear sampling and circular means
# --------------------------------------------------------------------------

def test_bilinear_reproduces_pixels_and_zero_outside(orc):
    n = 16
    f = inputs.random_image(n, seed=5)
    x = inputs.pixel_centres(n)
    for iy in (0, 3, 15):
        for ix in (0, 7, 15):
            assert orc.bilinear(f, x[ix], x[iy]) == f[iy, ix]
    h = 2.0 / n
    assert orc.bilinear(f, -1.0 - h, 0.0) == 0.0  # more than half a pixel outside: zero
    assert orc.bilinear(f, 0.0, 1.0 + h) == 0.0
    # half a pixel outside the outer pixel centre: half of the edge pixel (zero outside)
    assert abs(orc.bilinear(f, x[0] - h / 2, x[5]) - 0.5 * f[5, 0]) < 1e-14


def test_circle_mean_exact_for_bilinear_functions(orc):
    """f = c0 + c1 x + c2 y + c3 x y is reproduced exactly by bilinear
    interpolation inside the grid, and the K-node trapezoid rule (K >= 3)
    integrates cos, sin and sin(2 phi) exactly: the circle mean is f(centre)."""
    n = 32
    x = inputs.pixel_centres(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    c = (0.3, -1.2, 0.7, 2.5)
    f = c[0] + c[1] * X + c[2] * Y + c[3] * X * Y
    rng = np.random.default_rng(7)
    for K in (3, 5, 16, 129):
        for _ in range(4):
            cx, cy = rng.uniform(-0.4, 0.4, 2)
            r = rng.uniform(0.0, 0.45)
            ref = c[0] + c[1] * cx + c[2] * cy + c[3] * cx * cy
            assert abs(orc.circle_mean(f, cx, cy, r, K) - ref) < 1e-13


def test_circle_mean_gaussian_closed_form(orc):
    """Mean of exp(-|x|^2/s^2) over the circle of radius r about a point at
    distance rho: exp(-(rho^2 + r^2)/s^2) I0(2 rho r / s^2).  Converges at
    second order in h (bilinear interpolation) for large K."""
    s = 0.3
    cases = [(0.5, 0.2), (0.1, 0.6), (0.7, 0.35)]
    errs = []
    for n in (32, 64, 128):
        x = inputs.pixel_centres(n)
        X, Y = np.meshgrid(x, x, indexing="xy")
        f = np.exp(-(X ** 2 + Y ** 2) / s ** 2)
        e = 0.0
        for rho, r in cases:
            ref = math.exp(-((rho - r) ** 2) / s ** 2) * special.i0e(2 * rho * r / s ** 2)
            e = max(e, abs(orc.circle_mean(f, rho, 0.0, r, 4096) - ref))
        errs.append(e)
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
    assert errs[-1] < 2e-4


def test_detector_convention_matches_paper_arcs(orc):
    """Cell-centred detectors: n detectors with the pitch of the full array
    cover n * pitch; 170 and 112 of 256-on-270-degrees give the printed
    179.30 and 118.125 degrees (Sec. 2.1, Sec. 2.4.2)."""
    with open(os.path.join(GOLDEN, "detector_arcs.json")) as fh:
        gold = json.load(fh)
    n_full, span = gold["n_full"], math.radians(gold["span_full_deg"])
    g = geom(orc, 64, n_full, 16, 16, span=span)
    xy = orc.detectors(g)
    theta = np.unwrap(np.arctan2(xy[:, 1], xy[:, 0]))
    pitch = np.diff(theta)
    assert np.allclose(pitch, span / n_full, atol=1e-12)
    assert abs(theta[0] - span / n_full / 2) < 1e-12  # first detector half a pitch in
    for sub in gold["subsets"]:
        cover = math.degrees(sub["n_det"] * pitch.mean())
        assert round(cover, sub["printed_decimals"]) == pytest.approx(sub["coverage_deg"], abs=1e-12)
        gs = geom(orc, 64, sub["n_det"], 16, 16, span=math.radians(cover))
        th_s = np.unwrap(np.arctan2(orc.detectors(gs)[:, 1], orc.detectors(gs)[:, 0]))
        assert np.allclose(th_s, theta[: sub["n_det"]], atol=1e-12)


# --------------------------------------------------------------------------
# Whole operator
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,n_det,n_t,K,span", [(8, 5, 12, 7, 2 * math.pi), (32, 16, 48, 40, math.pi),
                                                 (20, 9, 30, 33, 1.5 * math.pi)])
def test_adjoint_identity(orc, n, n_det, n_t, K, span):
    g = geom(orc, n, n_det, n_t, K, span=span, start=0.3)
    f = inputs.random_image(n, seed=1)
    d = inputs.random_data(n_det, n_t, seed=2)
    Af = orc.forward(g, f)
    Atd = orc.adjoint(g, d)
    lhs, rhs = float(np.sum(Af * d)), float(np.sum(f * Atd))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Af) * np.linalg.norm(d)
    # the two stages separately
    M = orc.circular_means(g, f)
    Mb = inputs.random_data(n_det, n_t + 2, seed=3)
    assert abs(np.sum(M * Mb) - np.sum(f * orc.adjoint_means(g, Mb))) <= 1e-12 * np.linalg.norm(M) * np.linalg.norm(Mb)


def _dense_bruteforce(n, n_det, n_t, K, T, start, span):
    """Independent dense build of A: per-sample footprints enumerated in numpy
    and the Abel weights from QUADPACK (not the oracle's closed form)."""
    h = 2.0 / n
    n_r = n_t + 2
    d = T / n_t
    C = np.zeros((n_det * n_r, n * n))
    for j in range(n_det):
        th = start + (j + 0.5) * span / n_det
        for m in range(n_r):
            for q in range(K):
                ph = 2 * math.pi * q / K
                sx, sy = math.cos(th) + m * d * math.cos(ph), math.sin(th) + m * d * math.sin(ph)
                u, v = (sx + 1) / h - 0.5, (sy + 1) / h - 0.5
                i0, j0 = math.floor(u), math.floor(v)
                a, b = u - i0, v - j0
                for di, dj, w in ((0, 0, (1 - a) * (1 - b)), (1, 0, a * (1 - b)), (0, 1, (1 - a) * b), (1, 1, a * b)):
                    ii, jj = i0 + di, j0 + dj
                    if 0 <= ii < n and 0 <= jj < n:
                        C[j * n_r + m, jj * n + ii] += w / K
    Pq = np.zeros((n_t, n_r))
    for k in range(1, n_t + 1):
        for m in range(n_r):
            Pq[k - 1, m] = _w_quad(k + 0.5, m) - _w_quad(k - 0.5, m)
    A = np.zeros((n_det * n_t, n * n))
    for j in range(n_det):
        A[j * n_t:(j + 1) * n_t] = Pq @ C[j * n_r:(j + 1) * n_r]
    return A


@pytest.mark.slow
def test_dense_bruteforce_tiny(orc):
    n, n_det, n_t, K, T, start, span = 6, 3, 8, 7, 2.0, 0.2, 1.7 * math.pi
    g = geom(orc, n, n_det, n_t, K, span=span, start=start, t_max=T)
    A = np.zeros((n_det * n_t, n * n))
    for i in range(n * n):
        e = np.zeros(n * n)
        e[i] = 1.0
        A[:, i] = orc.forward(g, e.reshape(n, n)).ravel()
    ref = _dense_bruteforce(n, n_det, n_t, K, T, start, span)
    assert np.max(np.abs(A - ref)) <= 1e-12 * np.max(np.abs(ref))
    # adjoint = transpose, column by column
    for r in range(0, n_det * n_t, 5):
        e = np.zeros(n_det * n_t)
        e[r] = 1.0
        assert np.allclose(orc.adjoint(g, e.reshape(n_det, n_t)).ravel(), A[r], atol=1e-13, rtol=0)


def _hankel_trace(s, t):
    """Exact 2D wave solution at |x| = 1 for p(x,0) = exp(-|x|^2/s^2), p_t(x,0) = 0:
    p = (s^2/2) int_0^inf exp(-s^2 k^2/4) J0(k) cos(k t) k dk."""
    kmax = 2.0 * math.sqrt(40.0) / s
    f = lambda k: math.exp(-s * s * k * k / 4) * special.j0(k) * math.cos(k * t) * k
    return s * s / 2 * integrate.quad(f, 0.0, kmax, limit=2000, epsabs=1e-14, epsrel=1e-12)[0]


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
def test_forward_converges_to_wave_solution(orc):
    """The whole discrete A (means + Abel + midpoint derivative, detector
    radius 1, times k Delta) converges to the exact solution of Eq. (1)
    observed by Eq. (2), at second order."""
    s = 0.2
    errs = []
    for n, n_t, K in ((64, 128, 256), (128, 256, 512), (256, 512, 1024)):
        g = geom(orc, n, 1, n_t, K, start=0.3)
        x = inputs.pixel_centres(n)
        X, Y = np.meshgrid(x, x, indexing="xy")
        out = orc.forward(g, np.exp(-(X ** 2 + Y ** 2) / s ** 2))[0]
        t = np.arange(1, n_t + 1) * 2.0 / n_t
        ref = np.array([_hankel_trace(s, tt) for tt in t])
        errs.append(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs
    assert errs[-1] < 1e-3


# --------------------------------------------------------------------------
# TV
# --------------------------------------------------------------------------

def test_tv_closed_forms(orc):
    n, eps = 12, 1e-3
    v, gr = orc.tv(np.full((n, n), 3.0), eps)
    assert abs(v - n * n * eps) < 1e-15 and np.all(gr == 0)
    a = 0.25
    ramp = np.tile(a * np.arange(n), (n, 1))  # f[i][j] = a j
    v, gr = orc.tv(ramp, eps)
    s = math.sqrt(a * a + eps * eps)
    assert abs(v - (n * (n - 1) * s + n * eps)) < 1e-12
    assert np.allclose(gr[:, 0], -a / s) and np.allclose(gr[:, -1], a / s) and np.allclose(gr[:, 1:-1], 0, atol=1e-14)


def test_tv_gradient_finite_differences(orc):
    n, eps = 9, 0.05
    f = inputs.random_image(n, seed=9)
    _, gr = orc.tv(f, eps)
    hstep = 1e-6
    for (i, j) in [(0, 0), (4, 4), (8, 8), (0, 8), (8, 0), (3, 7)]:
        fp, fm = f.copy(), f.copy()
        fp[i, j] += hstep
        fm[i, j] -= hstep
        fd = (orc.tv(fp, eps, with_grad=False) - orc.tv(fm, eps, with_grad=False)) / (2 * hstep)
        assert abs(fd - gr[i, j]) <= 1e-7 * max(1.0, abs(gr[i, j]))


def test_threads_do_not_change_forward(orc):
    g = geom(orc, 32, 12, 40, 48, span=math.pi)
    f = inputs.gaussian_phantom(32, 5, seed=1)
    orc.set_threads(1)
    a = orc.forward(g, f)
    b1 = orc.adjoint(g, a)
    orc.set_threads(4)
    b = orc.forward(g, f)
    b4 = orc.adjoint(g, a)
    orc.set_threads(1)
    assert np.array_equal(a, b)
    assert np.allclose(b1, b4, rtol=1e-14, atol=1e-15)


# --------------------------------------------------------------------------
# Symmetry of the whole operator under a quarter turn
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,n_det,K,start", [(24, 16, 32, 0.0), (17, 12, 20, 0.37), (32, 8, 64, 1.1)])
def test_quarter_turn_equivariance(orc, n, n_det, K, start):
    """Pixel (iy, ix) sits at (-1 + (ix+1/2)h, -1 + (iy+1/2)h) and detector j at
    angle start + (j+1/2) 2 pi / n_det counter-clockwise from +x.  np.rot90
    moves the content at (x, y) to (y, -x), a clockwise quarter turn about the
    centre, under which the pixel grid and (with K divisible by 4) the angular
    nodes map onto themselves.  So on a full circle with n_det divisible by 4,
    A(rot90 f) is A f with the detector rows moved back by n_det/4, and A^T
    commutes with the same pair of maps.  Catches swapped x/y, a mirrored
    axis or a wrong detector orientation."""
    g = geom(orc, n, n_det, 3 * n // 2, K, start=start)
    f = inputs.random_image(n, seed=21).astype(np.float64)
    a = orc.forward(g, f)
    b = orc.forward(g, np.rot90(f, 1))
    assert np.abs(b - np.roll(a, -n_det // 4, axis=0)).max() <= 1e-12 * np.abs(a).max()
    assert np.abs(b - np.roll(a, n_det // 4, axis=0)).max() > 1e-3 * np.abs(a).max()   # not symmetric by chance
    d = inputs.random_data(n_det, 3 * n // 2, seed=22).astype(np.float64)
    fa = orc.adjoint(g, d)
    fb = orc.adjoint(g, np.roll(d, -n_det // 4, axis=0))
    assert np.abs(fb - np.rot90(fa, 1)).max() <= 1e-12 * np.abs(fa).max()

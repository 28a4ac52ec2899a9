"""GPU parity of the primal-dual (Chambolle-Pock) TV iteration for Eq. (4).

``pat_pdhg_step`` runs through the C ABI and is compared with the FP64
oracle's iteration (``oracle/pdhg.py`` driven by the oracle's A and A^T) on the
same seeded data, iterate by iterate.

Tolerance: every map of the iteration except A and A^T (the two proximal maps,
the gradient and its transpose, the extrapolation) is evaluated to FP32
rounding, and A, A^T meet 1e-5 relative L2.  The iteration map is
non-expansive, so the deviation grows at most additively: after k iterations
each variable is within k * 1e-5 of the FP64 iterate, relative to its norm.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import pdhg as OP
from paper_2604_19176_gb300 import Geometry, PatPlan, inputs
from paper_2604_19176_gb300.recon import pdhg_reconstruct

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


def og(g: Geometry) -> O.Geometry:
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _data(g: Geometry, seed: int, noise: float = 0.02):
    f = inputs.vessel_phantom(g.n, seed=seed)
    d = inputs.add_noise(O.forward(og(g), f), noise, seed=seed + 1)
    return d.astype(np.float32).astype(np.float64)


def _oracle_norm_sq(g: Geometry, iters: int = 30) -> float:
    x = np.random.default_rng(0).random((g.n, g.n))
    lam = 0.0
    for _ in range(iters):
        y = O.adjoint(og(g), O.forward(og(g), x))
        lam = float(np.linalg.norm(y))
        x = y / lam
    return lam


def _gpu_state(plan, dev):
    z = lambda s: torch.zeros(s, dtype=torch.float32, device=dev)  # noqa: E731
    return {"f": z(plan.image_shape()), "fbar": z(plan.image_shape()), "y": z(plan.data_shape()),
            "px": z(plan.image_shape()), "py": z(plan.image_shape())}


@pytest.mark.parametrize("nonneg,beta", [(True, 0.0), (False, 0.0), (False, 200.0)])
def test_pdhg_iterates_match_oracle(cuda_dev, nonneg, beta):
    """beta > 0 is the mouse-data variant: no f >= 0, mean-intensity penalty
    beta/2 (mean f - 0.2)^2."""
    g = Geometry(64, 48, 0.3, 1.5 * math.pi, 96, 2.0, 128)
    data = _data(g, seed=5)
    s = 0.99 / math.sqrt(_oracle_norm_sq(g) + 8.0)
    alpha = 1e-3
    plan = PatPlan(g, device=cuda_dev)
    st = _gpu_state(plan, cuda_dev)
    gd = torch.tensor(data, dtype=torch.float32, device=cuda_dev)
    delta = torch.zeros(2, device=cuda_dev)
    fmean = torch.zeros(1, device=cuda_dev)
    ost = None
    A = lambda f: O.forward(og(g), f)  # noqa: E731
    At = lambda y: O.adjoint(og(g), y)  # noqa: E731
    mp = (beta, 0.2) if beta > 0 else None
    for k in range(12):
        plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, s, s, alpha, nonneg=nonneg, delta=delta,
                       beta=beta, mean_target=0.2, fmean=fmean if beta > 0 else None)
        ost, orel = OP.pdhg(A, At, data, g.n, alpha, s, s, 1, nonneg=nonneg, state=ost, mean_penalty=mp)
        torch.cuda.synchronize()
        if beta > 0:
            assert abs(float(fmean) - ost["f"].mean()) <= (k + 1) * OP_TOL * np.sqrt(np.mean(ost["f"] ** 2))
        tol = (k + 1) * OP_TOL
        for name in ("f", "fbar", "y"):
            assert rel(st[name].double().cpu().numpy(), ost[name]) <= tol, (k, name)
        if k > 0:   # p is zero after the first step (fbar = 0 there)
            p_gpu = np.stack([st["px"].double().cpu().numpy(), st["py"].double().cpu().numpy()])
            assert rel(p_gpu, np.stack([ost["px"], ost["py"]])) <= tol, (k, "p")
        d = delta.double().cpu().numpy()
        assert abs(math.sqrt(d[0] / d[1]) - orel[0]) <= tol * orel[0] + 1e-7, k
        if nonneg:
            assert float(st["f"].min()) >= 0.0


def test_pdhg_batched_uneven_instances(cuda_dev):
    """Two instances of different size and arc in one plan: each instance's
    iterates follow the oracle run on that instance alone."""
    geoms = [Geometry(64, 48, 0.3, 1.5 * math.pi, 96, 2.0, 128), Geometry(48, 40, 1.0, math.pi, 80, 2.0, 96)]
    datas = [_data(geoms[0], seed=5), _data(geoms[1], seed=7)]
    s, alpha = 0.3, 2e-3
    plan = PatPlan(geoms, device=cuda_dev)
    st = _gpu_state(plan, cuda_dev)
    fo, go = plan.layout()
    gd = torch.tensor(np.concatenate([d.ravel() for d in datas]), dtype=torch.float32, device=cuda_dev)
    delta = torch.zeros(4, device=cuda_dev)
    iters = 8
    for _ in range(iters):
        plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, s, s, alpha, delta=delta)
    torch.cuda.synchronize()
    f_all = st["f"].double().cpu().numpy().ravel()
    y_all = st["y"].double().cpu().numpy().ravel()
    for i, g in enumerate(geoms):
        ost, orel = OP.pdhg(lambda f: O.forward(og(g), f), lambda y: O.adjoint(og(g), y), datas[i], g.n, alpha, s, s,
                            iters)
        assert rel(f_all[fo[i]:fo[i + 1]].reshape(g.n, g.n), ost["f"]) <= iters * OP_TOL
        assert rel(y_all[go[i]:go[i + 1]].reshape(g.n_det, g.n_t), ost["y"]) <= iters * OP_TOL
        d = delta.double().cpu().numpy()[2 * i:2 * i + 2]
        assert abs(math.sqrt(d[0] / d[1]) - orel[-1]) <= iters * OP_TOL * orel[-1] + 1e-7


def test_pdhg_stop_rule_matches_oracle(cuda_dev):
    """Run to the relative-change rule of Sec. 2.3 (1e-4): the GPU stops at
    the oracle's iteration (within 2) and its image is the oracle's there."""
    g = Geometry(64, 48, 0.3, 1.5 * math.pi, 96, 2.0, 128)
    data = _data(g, seed=5)
    s = 0.99 / math.sqrt(_oracle_norm_sq(g) + 8.0)
    alpha = 1e-2
    plan = PatPlan(g, device=cuda_dev)
    f, hist, _ = pdhg_reconstruct(plan, torch.tensor(data, dtype=torch.float32, device=cuda_dev), alpha, iters=400,
                                  sigma=s, tau=s)
    k_gpu = hist[-1][0]
    assert hist[-1][1] <= 1e-4 and all(r > 1e-4 for k, r in hist[1:-1])
    A = lambda x: O.forward(og(g), x)  # noqa: E731
    At = lambda y: O.adjoint(og(g), y)  # noqa: E731
    O.set_threads(8)
    try:
        st, orel = OP.pdhg(A, At, data, g.n, alpha, s, s, k_gpu + 1)
        _, orel2 = OP.pdhg(A, At, data, g.n, alpha, s, s, 2, state=st)
    finally:
        O.set_threads(1)
    k_orc = next(k for k, r in enumerate(orel + orel2) if k > 0 and r <= 1e-4)
    assert abs(k_gpu - k_orc) <= 2
    assert rel(f.double().cpu().numpy(), st["f"]) <= 1e-3


def test_pdhg_mouse_variant_reconstruct(cuda_dev):
    """pdhg_reconstruct with nonneg=False and the mean penalty: the mean it
    keeps on the device is the image's mean, the penalty pulls the mean towards
    its target, and the iterates follow the oracle."""
    g = Geometry(64, 48, 0.3, 1.5 * math.pi, 96, 2.0, 128)
    data = _data(g, seed=5)
    plan = PatPlan(g, device=cuda_dev)
    gd = torch.tensor(data, dtype=torch.float32, device=cuda_dev)
    s = 0.99 / math.sqrt(_oracle_norm_sq(g) + 8.0)
    iters = 30
    f0, _, _ = pdhg_reconstruct(plan, gd, 1e-3, iters=iters, sigma=s, tau=s, nonneg=False, stop_tol=0.0)
    f1, _, st = pdhg_reconstruct(plan, gd, 1e-3, iters=iters, sigma=s, tau=s, nonneg=False,
                                 mean_penalty=(400.0, 0.5), stop_tol=0.0)
    assert abs(float(st["fmean"]) - float(f1.mean())) <= 1e-6 * float(f1.abs().max())
    assert abs(float(f1.mean()) - 0.5) < abs(float(f0.mean()) - 0.5)
    ost, _ = OP.pdhg(lambda x: O.forward(og(g), x), lambda y: O.adjoint(og(g), y), data, g.n, 1e-3, s, s, iters,
                     nonneg=False, mean_penalty=(400.0, 0.5))
    assert rel(f1.double().cpu().numpy(), ost["f"]) <= iters * OP_TOL


def test_pdhg_argument_checks(cuda_dev):
    from paper_2604_19176_gb300._lib import PatError

    g = Geometry(32, 16, 0.0, math.pi, 32, 2.0, 32)
    plan = PatPlan(g, device=cuda_dev)
    st = _gpu_state(plan, cuda_dev)
    gd = torch.zeros(plan.data_shape(), device=cuda_dev)
    with pytest.raises(PatError):   # f and fbar alias
        plan.pdhg_step(st["f"], st["f"], st["y"], st["px"], st["py"], gd, 0.1, 0.1, 1e-3)
    with pytest.raises(PatError):   # y is g
        plan.pdhg_step(st["f"], st["fbar"], gd, st["px"], st["py"], gd, 0.1, 0.1, 1e-3)
    with pytest.raises(PatError):   # non-positive step
        plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, 0.0, 0.1, 1e-3)
    with pytest.raises(PatError):   # negative weight
        plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, 0.1, 0.1, -1.0)
    with pytest.raises(PatError):   # mean penalty without the mean buffer
        plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, 0.1, 0.1, 1e-3, beta=1.0)
    with pytest.raises(PatError):   # delta inside f
        plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, 0.1, 0.1, 1e-3,
                       delta=st["f"].view(-1)[:2])
    with pytest.raises(PatError):   # mean buffer inside f
        plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, 0.1, 0.1, 1e-3, beta=1.0,
                       fmean=st["f"].view(-1)[:1])
    bf = PatPlan(g, device=cuda_dev, image_dtype=torch.bfloat16)
    with pytest.raises(PatError):   # FP32 plans only
        bf.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, 0.1, 0.1, 1e-3)


def test_fine_grid_data_no_inverse_crime(cuda_dev):
    """Data simulated on a 2x finer grid (Sec. 2.4.1): the GPU's fine-grid data
    match the oracle's A on the fine grid and the finely rendered phantom, and
    differ from the coarse-grid data by a small but nonzero discretisation gap."""
    from paper_2604_19176_gb300 import workloads
    from paper_2604_19176_gb300.api import Geometry as G

    wl = workloads.Workload("vessel64_half", (G(64, 48, 0.0, math.pi, 128, 2.0, 128),), "test",
                            {"phantom": "vessel", "tubes": 6, "seeds": [3]})
    fine = workloads.simulate_fine_data(wl, 2, device=cuda_dev).double().cpu().numpy()
    fg = workloads.fine_geometries(wl, 2)[0]
    fp = workloads.fine_phantoms(wl, 2)[0]
    ref = O.forward(og(fg), fp.astype(np.float32).astype(np.float64))
    assert rel(fine, ref) <= 1e-5
    coarse = O.forward(og(wl.geometries[0]), wl.phantoms()[0])
    gap = rel(coarse, ref)
    assert 1e-4 < gap < 0.3


def test_pdhg_full_size_vessel256(cuda_dev):
    """The 256^2 limited-view workload (128 detectors on 180 degrees, 512 times,
    K 512) at full size, in the launch configuration the benchmark uses: three
    primal-dual iterations against the oracle's."""
    from paper_2604_19176_gb300.workloads import vessel256_half

    wl = vessel256_half()
    g = wl.geometries[0]
    plan = PatPlan(g, device=cuda_dev, tune=1)
    O.set_threads(16)
    try:
        f = wl.phantoms()[0]
        data = inputs.add_noise(O.forward(og(g), f), 0.05, seed=78).astype(np.float32).astype(np.float64)
        s, alpha, iters = 0.3, 1e-3, 3
        st = _gpu_state(plan, cuda_dev)
        gd = torch.tensor(data, dtype=torch.float32, device=cuda_dev)
        for _ in range(iters):
            plan.pdhg_step(st["f"], st["fbar"], st["y"], st["px"], st["py"], gd, s, s, alpha)
        torch.cuda.synchronize()
        ost, _ = OP.pdhg(lambda x: O.forward(og(g), x), lambda y: O.adjoint(og(g), y), data, g.n, alpha, s, s, iters)
    finally:
        O.set_threads(1)
    for name in ("f", "y"):
        assert rel(st[name].double().cpu().numpy(), ost[name]) <= iters * OP_TOL, name
    p_gpu = np.stack([st["px"].double().cpu().numpy(), st["py"].double().cpu().numpy()])
    assert rel(p_gpu, np.stack([ost["px"], ost["py"]])) <= iters * OP_TOL

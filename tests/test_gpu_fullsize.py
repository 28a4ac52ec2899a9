"""GPU parity at the full sizes the benchmark reports, against the FP64 oracle.

The oracle cannot run these workloads whole in seconds, so each check runs
the GPU on the full geometry and the oracle on a subset of its detectors:
a contiguous run of detectors j0 .. j0 + s - 1 of an arc is itself an arc
(start theta0 + j0 Phi / n_det, span s Phi / n_det, s detectors) with exactly
the same detector angles, time grid and angular rule.
  - forward: rows j0 .. j0 + s - 1 of the GPU's A f against the oracle's A f
    on the subset geometry;
  - adjoint: the GPU's A^T g for data that is zero outside those rows against
    the oracle's A^T of the subset geometry applied to those rows.
Workloads: 512^2 (256 detectors / 180 deg, n_t 1024, K 1024), the 760^2
experimental geometry (256 detectors / 270 deg, n_t 2030, K 1520), and
8 x 1024^2 (512 detectors / 270 deg, n_t 2048, K 2048) in FP32 and BF16 with
the autotuned tile, whose adjoint code word uses all 32 bits.
Tolerances as in test_gpu_parity: relative L2 <= 1e-5 (FP32 and BF16 storage
against the oracle on the BF16-rounded image), <= 4e-3 for BF16 against the
FP32 image.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_19176_gb300 import PatPlan, inputs, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-5


def sub_geometry(g, j0: int, s: int) -> O.Geometry:
    step = g.arc_span / g.n_det
    return O.Geometry(g.n, s, g.arc_start + j0 * step, s * step, g.n_t, g.t_max, g.n_angles)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def subsets(n_det: int, s: int = 4):
    return [(0, s), (n_det // 2 - s // 2, s), (n_det - s, s)]


@pytest.fixture(autouse=True)
def _oracle_threads():
    O.set_threads(8)
    yield
    O.set_threads(1)


def check_single(plan, g, f, dev, tol=TOL):
    """Forward rows and adjoint of data on three detector subsets."""
    fr = torch.tensor(f, dtype=plan.image_dtype, device=dev)
    f_in = fr.double().cpu().numpy()          # what the GPU sees (BF16-rounded for BF16 plans)
    gf = plan.forward(fr).double().cpu().numpy()
    for j0, s in subsets(g.n_det):
        sg = sub_geometry(g, j0, s)
        assert rel(gf[j0:j0 + s], O.forward(sg, f_in)) <= tol, (j0, s)
        d = inputs.random_data(s, g.n_t, seed=500 + j0).astype(np.float32)
        full = torch.zeros(g.n_det, g.n_t, dtype=torch.float32, device=dev)
        full[j0:j0 + s] = torch.tensor(d, device=dev)
        fa = plan.adjoint(full).double().cpu().numpy()
        assert rel(fa, O.adjoint(sg, d.astype(np.float64))) <= tol, (j0, s)


def test_vessel512_half_full_size(cuda_dev):
    wl = workloads.vessel512_half()
    g = wl.geometries[0]
    plan = PatPlan(g, device=cuda_dev, tune=1)
    check_single(plan, g, wl.phantoms()[0].astype(np.float32), cuda_dev)


def test_exp760_270_full_size(cuda_dev):
    wl = workloads.exp760_270()
    g = wl.geometries[0]
    plan = PatPlan(g, device=cuda_dev, tune=1)
    check_single(plan, g, wl.phantoms()[0].astype(np.float32), cuda_dev)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_vessel1024_b8_full_size(cuda_dev, dtype):
    """The 1024^2 x 8 precision-study workload in one plan with the autotuned
    tile: rows of A for instances 0 and 7, and an adjoint whose data is zero
    except for one detector subset in instance 0 and one in instance 7 (every
    other instance's image must come out exactly zero)."""
    wl = workloads.vessel1024_b8()
    geoms = list(wl.geometries)
    g = geoms[0]
    phs = np.stack(wl.phantoms()).astype(np.float32)
    plan = PatPlan(geoms, device=cuda_dev, image_dtype=dtype, tune=1)
    info = plan.info()
    if dtype == torch.float32:
        assert info["adj_mode"] == 1          # one-sample code lists: 9 + 12 + 11 = 32 bits per code (no pair bit)
    ft = torch.tensor(phs, dtype=dtype, device=cuda_dev)
    f_in = ft.double().cpu().numpy()
    gf = plan.forward(ft).double().cpu().numpy()
    picks = {0: (0, 4), 7: (g.n_det - 4, 4)}
    for i, (j0, s) in picks.items():
        sg = sub_geometry(g, j0, s)
        assert rel(gf[i, j0:j0 + s], O.forward(sg, f_in[i])) <= TOL, i
        if dtype == torch.bfloat16:
            assert rel(gf[i, j0:j0 + s], O.forward(sg, phs[i].astype(np.float64))) <= 4e-3, i
    data = torch.zeros(plan.data_shape(), dtype=torch.float32, device=cuda_dev)
    ds = {}
    for i, (j0, s) in picks.items():
        ds[i] = inputs.random_data(s, g.n_t, seed=600 + i).astype(np.float32)
        data[i, j0:j0 + s] = torch.tensor(ds[i], device=cuda_dev)
    fa = plan.adjoint(data)
    for i in range(len(geoms)):
        if i not in picks:
            assert not bool(fa[i].any()), i
    fa = fa.double().cpu().numpy()
    for i, (j0, s) in picks.items():
        ref = O.adjoint(sub_geometry(g, j0, s), ds[i].astype(np.float64))
        assert rel(fa[i], ref) <= (TOL if dtype == torch.float32 else 4e-3), i

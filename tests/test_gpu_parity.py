"""GPU parity: the CUDA operators (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 unless stated):
  FP32 forward / adjoint            <= 1e-5
  GPU adjoint identity              <= 1e-5
  BF16 image storage vs the oracle on the BF16-rounded image  <= 1e-5
  BF16 image storage vs the oracle on the FP32 image          <= 4e-3
Inputs are FP32-rounded before the oracle sees them, so the tolerance
measures the kernels' arithmetic, not the input rounding.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_19176_gb300 import Geometry, PatPlan, inputs
from paper_2604_19176_gb300.workloads import gauss64_full, vessel256_half

pytestmark = pytest.mark.gpu

TOL = 1e-5


def og(g: Geometry) -> O.Geometry:
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def run_fwd(plan, f, dev):
    out = plan.forward(torch.tensor(f, dtype=plan.image_dtype, device=dev))
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def run_adj(plan, g, dev):
    out = plan.adjoint(torch.tensor(g, dtype=torch.float32, device=dev))
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def test_forward_adjoint_gauss64(cuda_dev):
    wl = gauss64_full()
    g = wl.geometries[0]
    f = f32(wl.phantoms()[0])
    d = f32(inputs.random_data(g.n_det, g.n_t, seed=21))
    plan = PatPlan(g, device=cuda_dev)
    assert rel(run_fwd(plan, f, cuda_dev), O.forward(og(g), f)) <= TOL
    assert rel(run_adj(plan, d, cuda_dev), O.adjoint(og(g), d)) <= TOL


def test_forward_adjoint_vessel256_full_size(cuda_dev):
    """The benchmark geometry at full size, elementwise against the oracle."""
    O.set_threads(8)
    wl = vessel256_half()
    g = wl.geometries[0]
    f = f32(wl.phantoms()[0])
    d = f32(inputs.random_data(g.n_det, g.n_t, seed=22))
    plan = PatPlan(g, device=cuda_dev)
    gf = run_fwd(plan, f, cuda_dev)
    ref = O.forward(og(g), f)
    assert rel(gf, ref) <= TOL
    assert np.max(np.abs(gf - ref)) <= 2e-5 * np.max(np.abs(ref))
    fa = run_adj(plan, d, cuda_dev)
    refa = O.adjoint(og(g), d)
    assert rel(fa, refa) <= TOL
    assert np.max(np.abs(fa - refa)) <= 2e-5 * np.max(np.abs(refa))
    O.set_threads(1)


@pytest.mark.parametrize("kw", [dict(m_lanes=16), dict(m_lanes=8), dict(q_piece=4), dict(band_rows=5),
                                dict(band_rows=17, m_lanes=8, q_piece=12), dict(adj_groups=1, adj_mode=2), dict(adj_groups=3, adj_mode=2),
                                dict(adj_groups=16, adj_mode=2), dict(adj_mode=1), dict(adj_mode=1, adj_groups=3),
                                dict(adj_mode=3), dict(adj_mode=3, adj_groups=5), dict(adj_mode=4),
                                dict(adj_mode=4, adj_groups=3), dict(adj_mode=4, adj_jblock=1),
                                dict(adj_mode=1, adj_jblock=3), dict(adj_mode=4, adj_jblock=64, adj_groups=16),
                                dict(adj_mode=1, adj_jblock=5, adj_groups=7), dict(abel_split=1),
                                dict(abel_split=2), dict(abel_split=8), dict(tune=1)])
def test_tile_shapes_agree_with_oracle(cuda_dev, kw):
    g = Geometry(48, 24, 0.4, 1.3 * math.pi, 80, 2.0, 70)
    f = f32(inputs.gaussian_phantom(48, 5, seed=3) + 0.1 * inputs.random_image(48, seed=4))
    d = f32(inputs.random_data(g.n_det, g.n_t, seed=5))
    plan = PatPlan(g, device=cuda_dev, **kw)
    assert rel(run_fwd(plan, f, cuda_dev), O.forward(og(g), f)) <= TOL
    assert rel(run_adj(plan, d, cuda_dev), O.adjoint(og(g), d)) <= TOL


@pytest.mark.parametrize("g", [
    Geometry(8, 1, 0.0, 2 * math.pi, 1, 2.0, 3),        # smallest everything
    Geometry(8, 3, 1.0, 0.1, 5, 0.3, 4),                # tiny arc, short time range
    Geometry(12, 7, -2.0, 2 * math.pi, 33, 3.0, 9),     # radii reach beyond the image
    Geometry(64, 5, 0.7, 0.5 * math.pi, 17, 2.0, 1000), # K much larger than the radii count
    Geometry(100, 33, 0.0, 2 * math.pi, 150, 2.0, 31),  # N not a multiple of the tiles
])
def test_edge_geometries(cuda_dev, g):
    f = f32(inputs.random_image(g.n, seed=6))
    d = f32(inputs.random_data(g.n_det, g.n_t, seed=7))
    plan = PatPlan(g, device=cuda_dev)
    assert rel(run_fwd(plan, f, cuda_dev), O.forward(og(g), f)) <= TOL
    assert rel(run_adj(plan, d, cuda_dev), O.adjoint(og(g), d)) <= TOL


def test_adjoint_identity_gpu(cuda_dev):
    g = Geometry(96, 40, 0.2, 1.5 * math.pi, 128, 2.0, 150)
    plan = PatPlan(g, device=cuda_dev)
    f = torch.tensor(inputs.random_image(96, seed=8), dtype=torch.float32, device=cuda_dev)
    d = torch.tensor(inputs.random_data(g.n_det, g.n_t, seed=9), dtype=torch.float32, device=cuda_dev)
    Af = plan.forward(f)
    Atd = plan.adjoint(d)
    lhs = float((Af.double() * d.double()).sum())
    rhs = float((f.double() * Atd.double()).sum())
    assert abs(lhs - rhs) <= TOL * float(Af.double().norm() * d.double().norm())


def test_uneven_batch_and_identical_batch(cuda_dev):
    geoms = [Geometry(32, 16, 0.0, 2 * math.pi, 64, 2.0, 64),
             Geometry(48, 9, 0.5, 0.5 * math.pi, 40, 2.0, 96),
             Geometry(24, 30, 1.0, 1.5 * math.pi, 100, 2.5, 48),
             Geometry(32, 16, 0.0, 2 * math.pi, 64, 2.0, 64)]
    plan = PatPlan(geoms, device=cuda_dev)
    fo, go = plan.layout()
    imgs = [f32(inputs.random_image(gg.n, seed=10 + i)) for i, gg in enumerate(geoms)]
    datas = [f32(inputs.random_data(gg.n_det, gg.n_t, seed=20 + i)) for i, gg in enumerate(geoms)]
    flat_f = np.concatenate([x.ravel() for x in imgs])
    flat_g = np.concatenate([x.ravel() for x in datas])
    out_g = run_fwd(plan, flat_f, cuda_dev)
    out_f = run_adj(plan, flat_g, cuda_dev)
    for i, gg in enumerate(geoms):
        assert rel(out_g[go[i]:go[i + 1]].reshape(gg.n_det, gg.n_t), O.forward(og(gg), imgs[i])) <= TOL
        assert rel(out_f[fo[i]:fo[i + 1]].reshape(gg.n, gg.n), O.adjoint(og(gg), datas[i])) <= TOL
    # B identical instances: (B, N, N) -> (B, n_det, n_t)
    g = geoms[1]
    bplan = PatPlan([g] * 3, device=cuda_dev)
    fb = np.stack([f32(inputs.random_image(g.n, seed=30 + i)) for i in range(3)])
    ob = run_fwd(bplan, fb, cuda_dev)
    assert ob.shape == (3, g.n_det, g.n_t)
    for i in range(3):
        assert rel(ob[i], O.forward(og(g), fb[i])) <= TOL


def test_bf16_storage_bounds(cuda_dev):
    g = Geometry(128, 64, 0.0, 1.5 * math.pi, 256, 2.0, 256)
    f = inputs.mixed_phantom(128, 12, 5, seed=11)
    fb = torch.tensor(f, dtype=torch.bfloat16)
    f_b = fb.double().numpy()
    plan = PatPlan(g, device=cuda_dev, image_dtype=torch.bfloat16)
    out = plan.forward(fb.to(cuda_dev))
    torch.cuda.synchronize()
    out = out.double().cpu().numpy()
    assert rel(out, O.forward(og(g), f_b)) <= TOL
    assert rel(out, O.forward(og(g), f)) <= 4e-3
    d = f32(inputs.random_data(g.n_det, g.n_t, seed=12))
    fa = plan.adjoint(torch.tensor(d, dtype=torch.float32, device=cuda_dev))
    torch.cuda.synchronize()
    assert fa.dtype == torch.bfloat16
    assert rel(fa.double().cpu().numpy(), O.adjoint(og(g), d)) <= 4e-3


def test_tv_value_and_gradient(cuda_dev):
    g = Geometry(72, 8, 0.0, math.pi, 16, 2.0, 16)
    plan = PatPlan([g, g], device=cuda_dev)
    f = np.stack([f32(inputs.vessel_phantom(72, 6, seed=13)), f32(inputs.random_image(72, seed=14))])
    val, grad = plan.tv_grad(torch.tensor(f, dtype=torch.float32, device=cuda_dev), 1e-2)
    torch.cuda.synchronize()
    for i in range(2):
        rv, rg = O.tv(f[i], 1e-2)
        assert abs(float(val[i]) - rv) <= 1e-5 * rv
        assert rel(grad[i].double().cpu().numpy(), rg) <= 1e-5


def test_tv_grad_refuses_overlapping_buffers(cuda_dev):
    """pat_tv_grad reads neighbouring pixels that other CTAs would already have
    overwritten in place: a gradient overlapping the images, or a value buffer
    inside either, is refused before anything is enqueued."""
    import ctypes

    from paper_2604_19176_gb300 import _lib

    lib = _lib.load()
    g = Geometry(64, 8, 0.0, math.pi, 16, 2.0, 16)
    plan = PatPlan([g, g], device=cuda_dev)
    f = torch.rand(2, 64, 64, device=cuda_dev)
    grad = torch.empty_like(f)
    val = torch.empty(2, device=cuda_dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(cuda_dev).cuda_stream)
    p = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + 4 * off)
    e = ctypes.c_float(1e-2)
    assert lib.pat_tv_grad(plan._h, p(f), e, p(f), p(val), stream) == 1           # in place
    assert lib.pat_tv_grad(plan._h, p(f), e, p(f, 64), p(val), stream) == 1       # shifted by one row
    assert lib.pat_tv_grad(plan._h, p(f), e, p(grad), p(f, 3), stream) == 1       # value inside the images
    assert lib.pat_tv_grad(plan._h, p(f), e, p(grad), p(grad, 8), stream) == 1    # value inside the gradient
    assert lib.pat_tv_grad(plan._h, p(f), e, p(grad), p(val), stream) == 0
    torch.cuda.synchronize()
    rv, rg = O.tv(f[1].double().cpu().numpy(), 1e-2)
    assert abs(float(val[1]) - rv) <= 1e-5 * rv
    assert rel(grad[1].double().cpu().numpy(), rg) <= 1e-5


def test_quarter_turn_equivariance_full_size(cuda_dev):
    """The quarter-turn symmetry of the oracle pin, through the GPU path at
    full size (256^2, 128 detectors on the full circle, n_t = K = 512): a
    clockwise quarter turn of the image (np.rot90) moves A f's detector rows
    back by n_det/4, and A^T commutes with the same maps.  The exact operator
    does so to rounding and each GPU evaluation is within the 1e-5 parity
    bound of it, so two evaluations differ by at most 2e-5."""
    g = Geometry(256, 128, 0.2, 2 * math.pi, 512, 2.0, 512)
    plan = PatPlan(g, device=cuda_dev)
    f = f32(inputs.vessel_phantom(256, 12, seed=31))
    fr = np.ascontiguousarray(np.rot90(f, 1))
    a = plan.forward(torch.tensor(f, dtype=torch.float32, device=cuda_dev)).double().cpu().numpy()
    b = plan.forward(torch.tensor(fr, dtype=torch.float32, device=cuda_dev)).double().cpu().numpy()
    assert rel(b, np.roll(a, -32, axis=0)) <= 2e-5
    d = f32(inputs.random_data(128, 512, seed=32))
    dr = np.ascontiguousarray(np.roll(d, -32, axis=0))
    fa = plan.adjoint(torch.tensor(d, dtype=torch.float32, device=cuda_dev)).double().cpu().numpy()
    fb = plan.adjoint(torch.tensor(dr, dtype=torch.float32, device=cuda_dev)).double().cpu().numpy()
    assert rel(fb, np.rot90(fa, 1)) <= 2e-5


def test_residual_and_descent_step(cuda_dev):
    g = Geometry(40, 10, 0.0, math.pi, 20, 2.0, 16)
    plan = PatPlan(g, device=cuda_dev)
    a = torch.randn(10, 20, device=cuda_dev)
    b = torch.randn(10, 20, device=cuda_dev)
    r = plan.residual(a, b, scale=2.0)
    assert torch.allclose(r, 2.0 * (a - b), rtol=1e-6, atol=1e-6)
    f = torch.rand(40, 40, device=cuda_dev) - 0.3
    adj = torch.randn(40, 40, device=cuda_dev)
    tvg = torch.randn(40, 40, device=cuda_dev)
    delta = torch.zeros(2, device=cuda_dev)
    f0 = f.clone()
    plan.descent_step(f, adj, tvg, tau=0.1, lam=0.5, nonneg=True, delta=delta)
    ref = torch.clamp(f0 - 0.1 * (adj + 0.5 * tvg), min=0)
    assert torch.allclose(f, ref, rtol=1e-6, atol=1e-6)
    assert abs(float(delta[0]) - float(((ref - f0) ** 2).sum())) <= 1e-4 * float(((ref - f0) ** 2).sum())
    assert abs(float(delta[1]) - float((ref ** 2).sum())) <= 1e-4 * float((ref ** 2).sum())


def test_deterministic_and_sample_count(cuda_dev):
    g = vessel256_half().geometries[0]
    plan = PatPlan(g, device=cuda_dev)
    f = torch.tensor(inputs.random_image(256, seed=15), dtype=torch.float32, device=cuda_dev)
    d = torch.tensor(inputs.random_data(g.n_det, g.n_t, seed=16), dtype=torch.float32, device=cuda_dev)
    a1, a2 = plan.forward(f), plan.forward(f).clone()
    b1, b2 = plan.adjoint(d), plan.adjoint(d).clone()
    assert torch.equal(a1, a2) and torch.equal(b1, b2)
    info = plan.info()
    ref = O.count_samples(og(g))
    assert abs(info["samples"] - ref) <= 1e-4 * ref
    assert info["sample_slots"] >= info["samples"]


def test_plan_errors(cuda_dev):
    from paper_2604_19176_gb300._lib import PatError
    with pytest.raises(PatError):
        PatPlan(Geometry(10, 4, 0.0, math.pi, 8, 2.0, 8), device=cuda_dev)   # N not a multiple of 4
    with pytest.raises(PatError):
        PatPlan(Geometry(16, 4, 0.0, 7.0, 8, 2.0, 8), device=cuda_dev)    # arc beyond 2 pi
    plan = PatPlan(Geometry(16, 4, 0.0, math.pi, 8, 2.0, 8), device=cuda_dev)
    with pytest.raises(ValueError):
        plan.forward(torch.zeros(15, 16, device=cuda_dev))
    plan.close()


def test_fused_tv_step_matches_separate_calls(cuda_dev):
    """pat_tv_step with separate time-stage launches (time_pair = 1) equals
    pat_forward, pat_residual, pat_adjoint, pat_tv_grad and pat_descent_step
    in sequence (same arithmetic, fewer kernels).  The fused time stage sums
    its contractions in another order: tests/test_gpu_time_pair.py."""
    g = Geometry(64, 32, 0.2, math.pi, 96, 2.0, 128)
    plan = PatPlan(g, device=cuda_dev, time_pair=1)
    f0 = torch.tensor(np.abs(inputs.random_image(64, seed=41)), dtype=torch.float32, device=cuda_dev)
    data = torch.tensor(inputs.random_data(32, 96, seed=42), dtype=torch.float32, device=cuda_dev)
    tau, lam, eps = 0.05, 0.3, 1e-2
    # separate calls
    f_a = f0.clone()
    r = plan.residual(plan.forward(f_a), data)
    adj = plan.adjoint(r)
    _, tvg = plan.tv_grad(f_a, eps)
    da = torch.zeros(2, device=cuda_dev)
    plan.descent_step(f_a, adj, tvg, tau, lam, nonneg=True, delta=da)
    # fused
    f_b = torch.empty_like(f0)
    db = torch.zeros(2, device=cuda_dev)
    plan.tv_step(f0, f_b, data, tau, lam, eps, nonneg=True, delta=db)
    torch.cuda.synchronize()
    assert torch.equal(f_a, f_b)
    assert torch.equal(da, db)


def test_graphed_batched_uneven_forward_adjoint(cuda_dev):
    """Uneven instances in one plan, forward + adjoint captured in one CUDA
    graph: replays match the eager calls bitwise and the oracle."""
    from paper_2604_19176_gb300.graphs import GraphedOperator, GraphedTVStep
    from paper_2604_19176_gb300.workloads import batch64_uneven
    geoms = [Geometry(g.n // 4, g.n_det // 8, g.arc_start, g.arc_span, g.n_t // 8, g.t_max, g.n_angles // 4)
             for g in batch64_uneven().geometries[:12]]
    plan = PatPlan(geoms, device=cuda_dev)
    op = GraphedOperator(plan)
    fo, go = plan.layout()
    for rep in range(2):
        flat_f = np.concatenate([f32(inputs.random_image(g.n, seed=50 + 10 * rep + i)).ravel()
                                 for i, g in enumerate(geoms)])
        flat_g = np.concatenate([f32(inputs.random_data(g.n_det, g.n_t, seed=70 + 10 * rep + i)).ravel()
                                 for i, g in enumerate(geoms)])
        op.f_in.copy_(torch.tensor(flat_f, dtype=torch.float32))
        op.g_in.copy_(torch.tensor(flat_g, dtype=torch.float32))
        op.replay()
        torch.cuda.synchronize()
        eager_g = plan.forward(op.f_in)
        eager_f = plan.adjoint(op.g_in)
        torch.cuda.synchronize()
        assert torch.equal(op.g_out, eager_g) and torch.equal(op.f_out, eager_f)
    for i in (0, 5, 11):
        g = geoms[i]
        assert rel(op.g_out[go[i]:go[i + 1]].double().cpu().numpy().reshape(g.n_det, g.n_t),
                   O.forward(og(g), flat_f[fo[i]:fo[i + 1]].reshape(g.n, g.n))) <= TOL
    # graphed fused TV iterations equal eager ones
    g1 = Geometry(48, 24, 0.0, math.pi, 64, 2.0, 96)
    p1 = PatPlan(g1, device=cuda_dev)
    data = torch.tensor(inputs.random_data(24, 64, seed=80), dtype=torch.float32, device=cuda_dev)
    gt = GraphedTVStep(p1, data, 0.05, 0.1, 1e-2)
    gt.replay()
    gt.replay()
    f_e, tmp = torch.zeros(48, 48, device=cuda_dev), torch.zeros(48, 48, device=cuda_dev)
    for _ in range(2):
        p1.tv_step(f_e, tmp, data, 0.05, 0.1, 1e-2)
        p1.tv_step(tmp, f_e, data, 0.05, 0.1, 1e-2)
    torch.cuda.synchronize()
    assert torch.equal(gt.f, f_e)


def test_batch64_uneven_full_size_each_instance(cuda_dev):
    """Every instance of the 64-instance uneven batch (N up to 384, up to 512
    detectors and 1024 times, K = 2N) at full size, in one plan: forward on
    the seeded Gaussian + vessel phantoms, adjoint on white-noise data, each
    within 1e-5 of the oracle."""
    from paper_2604_19176_gb300.workloads import batch64_uneven
    wl = batch64_uneven()
    geoms = list(wl.geometries)
    plan = PatPlan(geoms, device=cuda_dev)
    fo, go = plan.layout()
    imgs = [f32(p) for p in wl.phantoms()]
    datas = [f32(inputs.random_data(g.n_det, g.n_t, seed=300 + i)) for i, g in enumerate(geoms)]
    flat_f = torch.tensor(np.concatenate([x.ravel() for x in imgs]), dtype=torch.float32, device=cuda_dev)
    flat_g = torch.tensor(np.concatenate([x.ravel() for x in datas]), dtype=torch.float32, device=cuda_dev)
    out_g = plan.forward(flat_f).double().cpu().numpy()
    out_f = plan.adjoint(flat_g).double().cpu().numpy()
    worst_f = worst_a = 0.0
    for i, g in enumerate(geoms):
        worst_f = max(worst_f, rel(out_g[go[i]:go[i + 1]].reshape(g.n_det, g.n_t), O.forward(og(g), imgs[i])))
        worst_a = max(worst_a, rel(out_f[fo[i]:fo[i + 1]].reshape(g.n, g.n), O.adjoint(og(g), datas[i])))
    assert worst_f <= TOL and worst_a <= TOL, (worst_f, worst_a)


def test_large_radius_positions_n384(cuda_dev):
    """N = 384 on the full circle (|coordinates| up to N/2, radii up to N):
    the split-form sample positions keep A and A^T within 1e-5 where plain
    FP32 positions do not."""
    g = Geometry(384, 48, 0.0, 2 * math.pi, 512, 2.0, 768)
    plan = PatPlan(g, device=cuda_dev)
    f = f32(inputs.random_image(384, seed=91))
    d = f32(inputs.random_data(48, 512, seed=92))
    assert rel(run_fwd(plan, f, cuda_dev), O.forward(og(g), f)) <= TOL
    assert rel(run_adj(plan, d, cuda_dev), O.adjoint(og(g), d)) <= TOL


def test_list_forms_agree_bitwise(cuda_dev):
    """Every list form holds the same samples in the order (j, q, m): one-sample
    codes, run-pair codes (a pair stands for radii m, m + 1 of one ray) at any
    detector block size, and fraction lists (the a, b that the codes
    recompute).  With one part per cell the moment sums then see the same
    terms in the same order (null entries add exact zeros), so the adjoints
    are bitwise equal."""
    g = Geometry(96, 40, 0.3, 1.5 * math.pi, 160, 2.0, 192)
    d = torch.tensor(inputs.random_data(40, 160, seed=61), dtype=torch.float32, device=cuda_dev)
    outs = []
    for mode, jb in ((3, 0), (1, 8), (1, 1000), (4, 8), (4, 3), (4, 1)):
        plan = PatPlan(g, device=cuda_dev, adj_mode=mode, adj_groups=1, adj_jblock=jb)
        inf = plan.info()
        assert inf["adj_mode"] == mode
        assert inf["adj_jblock"] == (jb if mode != 3 else 0)
        outs.append(plan.adjoint(d).clone())
    torch.cuda.synchronize()
    for o in outs[1:]:
        assert torch.equal(outs[0], o)


def test_run_pair_lists_split_in_parts(cuda_dev):
    """With several parts per patch the part boundaries fall at other samples
    for pair and one-sample codes; the adjoints then agree to FP32 rounding,
    and a pair code list is shorter than the one-sample list."""
    g = Geometry(96, 40, 0.3, 1.5 * math.pi, 160, 2.0, 192)
    d = torch.tensor(inputs.random_data(40, 160, seed=61), dtype=torch.float32, device=cuda_dev)
    p1 = PatPlan(g, device=cuda_dev, adj_mode=1, adj_groups=3, adj_jblock=8)
    p4 = PatPlan(g, device=cuda_dev, adj_mode=4, adj_groups=3, adj_jblock=8)
    a, b = p1.adjoint(d).double(), p4.adjoint(d).double()
    assert float((a - b).norm() / a.norm()) <= 1e-6
    assert p4.info()["list_bytes"] < 0.8 * p1.info()["list_bytes"]

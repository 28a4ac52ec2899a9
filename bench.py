"""Benchmark: A + A^T applications per second on the 256 x 256 limited-view workload.

One step is one projected-gradient TV iteration of the reconstruction
(Eq. (4)): g_pred = A f; r = g_pred - g; f_adj = A^T r; TV gradient;
f <- max(0, f - tau (f_adj + lam grad TV)).  That is one A and one A^T
application plus the TV term, all in the library's kernels.

Workload: N = 256 vessel phantom (12 tubes), 128 detectors on 180 degrees,
512 time samples on (0, 2], K = 512 angular nodes, measured data = A f + 1 %
noise.  Inputs are ~1.5 MB, far below the 129 MB L2, so L2 is flushed (a
256 MB buffer is written) before every timed step; each step is timed with
CUDA events on the launching stream and the flush lies outside the events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own image (weak scaling, no
collective on the data path); the time is the max over ranks.  The
reference arm (--impl reference) times the FP64 CPU oracle on the host
cores; it is the only other place this file runs the oracle.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "vessel256_half"
METRIC = "A+A^T applications/s (TV-gradient step, N=256, 128 det / 180 deg, n_t=512, K=512)"
UNIT = "applications/s"
LAM, EPS, NOISE = 1e-3, 1e-3, 0.01
SMEM_BYTES_PER_CLK_SM = 128        # shared-memory load bandwidth per SM per clock (32 banks x 4 B)
BYTES_PER_SAMPLE = 16              # 4 FP32 texels per bilinear sample
CLOCK_WINDOW_S = 0.5               # load before and after the timed steps while clocks are sampled


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--profile", action="store_true", help="short run for ncu captures (no flush, no extras)")
    p.add_argument("--tile", default="",
                   help="fixed tile shape m_lanes,q_piece,band_rows,adj_groups,adj_mode,abel_split[,tile_cols[,adj_jblock]] "
                        "instead of the autotuner (e.g. the tile_shape a previous run reported), for reproducible "
                        "profiles")
    return p.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's step time (every rank gets it); ranks run independent
    instances, so the job is as fast as its slowest rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def job_value(ms: float, world: int) -> float:
    """Whole-job throughput: one application per rank per step of `ms`."""
    return world * 1000.0 / ms


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash() -> str:
    """Hash of the library sources (kernels and the host code that lays out
    their tables), to invalidate stored ncu traffic after a change."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2604_19176_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if the
    kernel source has not changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash() or e.get("workload") != WORKLOAD:
        return None
    return e.get("bytes_per_launch")


def make_inputs(seed_offset: int = 0):
    from paper_2604_19176_gb300 import inputs
    from paper_2604_19176_gb300.workloads import vessel256_half

    wl = vessel256_half()
    g = wl.geometries[0]
    f_true = inputs.vessel_phantom(g.n, 12, seed=2 + seed_offset)
    return wl, g, f_true


def cpu_oracle_timing(g, f_true, budget_s: float = 12.0, threads: int = 0, max_reps: int = 50):
    """FP64 oracle A + A^T of the whole workload (every detector, no scaling)
    on the host cores (all of them, or ``threads``): as many applications as
    fit in about ``budget_s`` seconds (at least one)."""
    import oracle as O

    cores = threads if threads > 0 else (os.cpu_count() or 1)
    O.set_threads(cores)
    og = O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)
    d = np.random.default_rng(0).standard_normal((g.n_det, g.n_t))
    t0 = time.perf_counter()
    reps = 0
    while True:
        O.forward(og, f_true)
        O.adjoint(og, d)
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= max_reps:
            break
    dt = (time.perf_counter() - t0) / reps
    O.set_threads(1)
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} x (A + A^T) of the whole workload ({g.n_det} detectors, N={g.n}, n_t={g.n_t}, "
                      f"K={g.n_angles}); FP64, OpenMP over detectors, {cores} threads"}


def workload_config(g) -> dict:
    """The `config` object both arms print."""
    return {"workload": WORKLOAD, "N": g.n, "n_det": g.n_det, "arc_deg": 180, "n_t": g.n_t, "K": g.n_angles,
            "lambda": LAM, "tv_eps": EPS, "noise": "1% of max|g|",
            "l2": "flushed (256 MB write) before every timed step, outside the events",
            "step": "one A + A^T application (GPU: pat_tv_step: A f, residual, A^T r, TV gradient, update)"}


def reference_arm(args):
    """The FP64 oracle, as it stands, on the host cores: K steps after W
    warm-up steps, each step one whole A + A^T application of the workload
    (every detector), so the line's steps, metric and config are the GPU arm's."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O

    wl, g, f_true = make_inputs()
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    og = O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)
    d = np.random.default_rng(0).standard_normal((g.n_det, g.n_t))

    def step():
        O.forward(og, f_true)
        O.adjoint(og, d)

    for _ in range(args.warmup):
        step()
    per = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        per.append(time.perf_counter() - t0)
    O.set_threads(1)
    ms = 1000.0 * statistics.mean(per)
    val = 1000.0 / ms
    sample = (f"{args.steps} timed steps after {args.warmup} warm-up steps, each one A + A^T of the whole workload "
              f"({g.n_det} detectors); FP64, OpenMP over detectors, {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(g),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# secondary workloads (reported under "extras"; not the headline metric)
# --------------------------------------------------------------------------
def _time_steps(fn, stream, flush, steps, warmup=3):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for i in range(steps):
        if flush is not None:
            flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ms.append((a, b))
    torch.cuda.synchronize()
    return statistics.mean(x.elapsed_time(y) for x, y in ms)


def run_extras(dev, flush, with_oracle: bool = True) -> dict:
    import torch

    from paper_2604_19176_gb300 import PatPlan, inputs, workloads
    from paper_2604_19176_gb300.graphs import GraphedOperator
    from paper_2604_19176_gb300.recon import (UNet, operator_norm_sq, pat_apply, pdhg_reconstruct, pdhg_steps,
                                              tv_value)

    stream = torch.cuda.current_stream(dev)
    out = {}

    # DIP iteration: U-Net (4 levels, 32 base channels, FP32, no TF32) on the
    # 256^2 geometry, loss ||A f - g||^2 + 1e-4 TV(f), one Adam step at 1e-4.
    wl = workloads.vessel256_half()
    g = wl.geometries[0]
    plan = PatPlan(g, device=dev, tune=1)
    f_true = torch.tensor(wl.phantoms()[0], dtype=torch.float32, device=dev)
    data = plan.forward(f_true)
    torch.cuda.synchronize()
    data = torch.tensor(inputs.add_noise(data.double().cpu().numpy(), 0.05, seed=78), dtype=torch.float32,
                        device=dev)
    z = torch.tensor(inputs.dip_input(32, g.n, seed=3), dtype=torch.float32, device=dev)
    torch.manual_seed(0)
    net = UNet(in_ch=32, base=32).to(dev)
    opt = torch.optim.Adam(net.parameters(), lr=1e-4)

    def dip_iter():
        opt.zero_grad(set_to_none=True)
        f = net(z).reshape(g.n, g.n)
        r = pat_apply(f, plan) - data
        loss = (r * r).sum() + 1e-4 * tv_value(f, plan, 1e-3).sum()
        loss.backward()
        opt.step()

    it_ms = _time_steps(dip_iter, stream, flush, 20, warmup=5)
    plan.set_timing(True)
    for _ in range(10):
        dip_iter()
    torch.cuda.synchronize()
    plan.set_timing(False)
    kt = plan.kernel_times()
    op_ms = sum(v[0] for v in kt.values()) / 10
    out["dip_vessel256"] = {"iters_per_s": 1000.0 / it_ms, "ms_per_iter": it_ms, "operator_ms_per_iter": op_ms,
                            "operator_share": op_ms / it_ms,
                            "config": "U-Net 4 levels / 32 base channels FP32 (TF32 off), z ~ N(0, 0.1^2) "
                                      "1x32x256x256, Adam lr 1e-4, loss ||Af-g||^2 + 1e-4 TV, 5% noise"}

    # 512^2 variant, fused TV step
    wl = workloads.vessel512_half()
    g = wl.geometries[0]
    p512 = PatPlan(g, device=dev, tune=1)
    d512 = p512.forward(torch.tensor(wl.phantoms()[0], dtype=torch.float32, device=dev))
    fa, fb = torch.zeros(g.n, g.n, device=dev), torch.zeros(g.n, g.n, device=dev)
    ms512 = _time_steps(lambda: p512.tv_step(fa, fb, d512, 1e-4, 1e-3, 1e-3), stream, flush, 100)
    out["vessel512_half"] = {"apps_per_s": 1000.0 / ms512, "ms_per_step": ms512, "samples": p512.info()["samples"]}
    del p512

    # Primal-dual TV iteration (Eq. (4), the paper's baseline solver) on the
    # experimental-data geometry: 760^2, 256 detectors on 270 degrees, 2030 times.
    wl = workloads.exp760_270()
    g = wl.geometries[0]
    pp = PatPlan(g, device=dev, tune=1)
    dpd = pp.forward(torch.tensor(wl.phantoms()[0], dtype=torch.float32, device=dev))
    sp = 0.99 / math.sqrt(operator_norm_sq(pp, iters=10) + 8.0)
    stp = {k: torch.zeros(pp.data_shape() if k == "y" else pp.image_shape(), device=dev)
           for k in ("f", "fbar", "y", "px", "py")}
    msp = _time_steps(lambda: pp.pdhg_step(stp["f"], stp["fbar"], stp["y"], stp["px"], stp["py"], dpd, sp, sp, 1e-3),
                      stream, flush, 50, warmup=5)
    pp.set_timing(True)
    for _ in range(10):
        pp.pdhg_step(stp["f"], stp["fbar"], stp["y"], stp["px"], stp["py"], dpd, sp, sp, 1e-3)
    torch.cuda.synchronize()
    pp.set_timing(False)
    kt = {k: round(v[0] / v[1], 5) for k, v in pp.kernel_times().items() if v[1] > 0}
    out["pdhg_exp760_270"] = {"iters_per_s": 1000.0 / msp, "ms_per_iter": msp, "s_per_1000_iters": msp,
                              "samples": pp.info()["samples"], "kernels_per_iter": 6, "kernel_avg_ms": kt,
                              "context": "paper: 1000 primal-dual iterations in 130.5 s on an RTX A5000 "
                                         "(PyTorch, fast FFT-based A / A*), same geometry"}
    del pp, dpd, stp

    # TV reconstruction to the paper's stopping rule (relative change <= 1e-4,
    # Sec. 2.3) at 256^2 from data simulated on a 512^2 grid (no inverse crime,
    # Sec. 2.4.1) with 5% noise; primal-dual iterations, alpha = 1e-3.
    wl = workloads.vessel256_half()
    g = wl.geometries[0]
    pp = PatPlan(g, device=dev, tune=1)
    dfine = workloads.simulate_fine_data(wl, 2, device=dev)
    torch.cuda.synchronize()
    dfine = torch.tensor(inputs.add_noise(dfine.double().cpu().numpy(), 0.05, seed=79), dtype=torch.float32,
                         device=dev)
    sg, tg = pdhg_steps(pp)
    pdhg_reconstruct(pp, dfine, 1e-3, iters=20, sigma=sg, tau=tg, check_every=10)   # warm-up, not timed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f_rec, hist, _ = pdhg_reconstruct(pp, dfine, 1e-3, iters=5000, sigma=sg, tau=tg, check_every=10)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    f_true = torch.tensor(wl.phantoms()[0], dtype=torch.float32, device=dev)
    out["pdhg_vessel256_fine_data"] = {
        "iterations": hist[-1][0] + 1, "final_rel_change": hist[-1][1], "wall_s": wall,
        "rel_l2_error_vs_phantom": float((f_rec - f_true).norm() / f_true.norm()),
        "config": "data from A on 512^2 (K 1024) of the same analytic phantom, 5% noise; reconstruction 256^2, "
                  "alpha 1e-3, sigma = tau = 0.99/||K||, stop at relative change <= 1e-4 (tested every 10)"}
    del pp

    # BF16 image storage vs FP32 at 256^2 (forward + adjoint), errors vs the FP64 oracle
    wl = workloads.vessel256_half()
    g = wl.geometries[0]
    f_np = wl.phantoms()[0]
    rng_g = inputs.random_data(g.n_det, g.n_t, seed=5)
    res = {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        pp = PatPlan(g, device=dev, image_dtype=dt, tune=1)
        ft = torch.tensor(f_np, dtype=dt, device=dev)
        gt = torch.tensor(rng_g, dtype=torch.float32, device=dev)
        go, fo = torch.empty(pp.data_shape(), device=dev), torch.empty(pp.image_shape(), dtype=dt, device=dev)

        def fa_step():
            pp.forward(ft, out=go)
            pp.adjoint(gt, out=fo)

        res[name] = {"apps_per_s": 1000.0 / _time_steps(fa_step, stream, flush, 100)}
        fa_step()
        torch.cuda.synchronize()
        res[name]["_fwd"] = go.double().cpu().numpy()
        res[name]["_adj"] = fo.double().cpu().numpy()
    if with_oracle:
        import oracle as O

        O.set_threads(os.cpu_count() or 1)
        og = O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)
        ref_f = O.forward(og, f_np)
        ref_a = O.adjoint(og, rng_g.astype(np.float32).astype(np.float64))
        for name in res:
            res[name]["rel_l2_fwd_vs_fp64"] = float(np.linalg.norm(res[name]["_fwd"] - ref_f) / np.linalg.norm(ref_f))
            res[name]["rel_l2_adj_vs_fp64"] = float(np.linalg.norm(res[name]["_adj"] - ref_a) / np.linalg.norm(ref_a))
        O.set_threads(1)
    for name in res:
        res[name].pop("_fwd")
        res[name].pop("_adj")
    out["storage_256"] = res

    # 64 uneven instances, forward + adjoint replayed from one CUDA graph
    geoms = list(workloads.batch64_uneven().geometries)
    pb = PatPlan(geoms, device=dev, tune=1)
    op = GraphedOperator(pb)
    op.f_in.copy_(torch.rand(pb.image_shape(), device=dev))
    op.g_in.copy_(torch.rand(pb.data_shape(), device=dev))
    msb = _time_steps(op.replay, stream, flush, 20)
    out["batch64_uneven"] = {"instances_per_s": 64 * 1000.0 / msb, "ms_per_batch": msb,
                             "samples": pb.info()["samples"], "graph": "forward + adjoint, one replay"}
    del op, pb
    torch.cuda.empty_cache()
    out["precision_1024_b8"] = precision_study(dev, stream, flush, with_oracle)
    out["config_runs_256"] = config_runs(dev, stream)
    if with_oracle:
        out["oracle_cpu"] = oracle_cpu_table()
    return out


def config_runs(dev, stream) -> dict:
    """The reconstruction runs the 256^2 limited-view configurations name:
    500 fused projected-gradient TV iterations of Eq. (4) (lambda 1e-3,
    eps 1e-3, f >= 0) at 1 % and 5 % noise, and 2000 Adam steps (lr 1e-4)
    of the DIP loss of Eq. (5) (||A f - g||^2 + 1e-4 TV, 5 % noise, U-Net 4
    levels / 32 channels, z ~ N(0, 0.1^2)).  Reported: the final objective,
    the relative L2 error against the phantom, and the wall time."""
    import torch

    from paper_2604_19176_gb300 import PatPlan, inputs, workloads
    from paper_2604_19176_gb300.recon import UNet, operator_norm_sq, pat_apply, tv_value

    wl = workloads.vessel256_half()
    g = wl.geometries[0]
    f_np = wl.phantoms()[0]
    plan = PatPlan(g, device=dev, tune=1)
    f_true = torch.tensor(f_np, dtype=torch.float32, device=dev)
    clean = plan.forward(f_true).double().cpu().numpy()
    a2 = operator_norm_sq(plan)
    out = {}

    def objective(f, data, lam, eps, halve):
        r = plan.forward(f).double() - data.double()
        tv = float(plan.tv_value(f, eps)[0])
        return (0.5 if halve else 1.0) * float((r * r).sum()) + lam * tv

    for lvl, seed in ((0.01, 81), (0.05, 82)):
        data = torch.tensor(inputs.add_noise(clean, lvl, seed=seed), dtype=torch.float32, device=dev)
        tau = 1.0 / (a2 + 8.0 * LAM / EPS)
        fa, fb = torch.zeros_like(f_true), torch.zeros_like(f_true)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(250):
            plan.tv_step(fa, fb, data, tau, LAM, EPS, nonneg=True)
            plan.tv_step(fb, fa, data, tau, LAM, EPS, nonneg=True)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[f"tv500_noise{int(lvl * 100)}pct"] = {
            "iterations": 500, "wall_s": wall, "objective_final": objective(fa, data, LAM, EPS, True),
            "objective_initial": objective(torch.zeros_like(f_true), data, LAM, EPS, True),
            "rel_l2_error_vs_phantom": float((fa - f_true).norm() / f_true.norm()),
            "config": "Eq. (4): 1/2 ||A f - g||^2 + 1e-3 TV_eps (eps 1e-3), f >= 0, tau = 1/(||A||^2 + 8 lam/eps), "
                      "pat_tv_step from zero, data A f_true + noise at the stated fraction of max|g|"}

    data = torch.tensor(inputs.add_noise(clean, 0.05, seed=83), dtype=torch.float32, device=dev)
    z = torch.tensor(inputs.dip_input(32, g.n, seed=3), dtype=torch.float32, device=dev)
    torch.manual_seed(0)
    net = UNet(in_ch=32, base=32).to(dev)
    opt = torch.optim.Adam(net.parameters(), lr=1e-4)
    losses = torch.zeros(2000, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(2000):
        opt.zero_grad(set_to_none=True)
        f = net(z).reshape(g.n, g.n)
        r = pat_apply(f, plan) - data
        loss = (r * r).sum() + 1e-4 * tv_value(f, plan, 1e-3).sum()
        loss.backward()
        opt.step()
        losses[k] = loss.detach()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    with torch.no_grad():
        f = net(z).reshape(g.n, g.n)
    lc = losses.cpu().numpy()
    out["dip2000_noise5pct"] = {
        "steps": 2000, "wall_s": wall, "iters_per_s": 2000 / wall,
        "loss_first": float(lc[0]), "loss_min": float(lc.min()), "loss_last": float(lc[-1]),
        "loss_at": {str(k): float(lc[k]) for k in (0, 99, 499, 999, 1499, 1999)},
        "rel_l2_error_vs_phantom": float((f - f_true).norm() / f_true.norm()),
        "config": "Eq. (5): ||A f_theta - g||^2 + 1e-4 TV_eps (eps 1e-3), U-Net 4 levels / 32 base channels FP32 "
                  "(TF32 off), z ~ N(0, 0.1^2) 1x32x256x256, Adam lr 1e-4, 5 % noise"}
    del net, opt, plan
    torch.cuda.empty_cache()
    return out


def oracle_cpu_table() -> dict:
    """The FP64 oracle's A + A^T applications/s on the host, single-threaded and
    on all cores, for the 64^2 full-circle and the 256^2 limited-view workloads
    (bounded samples of a few seconds each; context, not a target)."""
    from paper_2604_19176_gb300 import workloads

    res = {}
    for wl in (workloads.gauss64_full(), workloads.vessel256_half()):
        g = wl.geometries[0]
        f = wl.phantoms()[0]
        one = cpu_oracle_timing(g, f, budget_s=3.0, threads=1)
        res[wl.name] = {"single_thread": one["value"], "sample_single": one["sample"]}
        if wl.name == "gauss64_full":
            allc = cpu_oracle_timing(g, f, budget_s=3.0)
            res[wl.name].update({"all_cores": allc["value"], "cores": allc["cores"]})
    res["unit"] = UNIT
    res["note"] = "vessel256_half on all cores is the cpu_baseline of this line"
    return res


def precision_study(dev, stream, flush, with_oracle: bool) -> dict:
    """BF16 vs FP32 image storage on the 1024^2 x 8 workload (forward + adjoint
    of the batch), with the error of each against the FP64 oracle on a 256^2
    replica: the same analytic phantom (same seed, same physical tube widths),
    the same 512 detectors on 270 degrees, time grid and angular rule."""
    import torch

    from paper_2604_19176_gb300 import Geometry, PatPlan, inputs, workloads

    wl = workloads.vessel1024_b8()
    geoms = list(wl.geometries)
    phs = np.stack(wl.phantoms())
    res = {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        pp = PatPlan(geoms, device=dev, image_dtype=dt, tune=1)
        ft = torch.tensor(phs, dtype=dt, device=dev)
        go = torch.empty(pp.data_shape(), device=dev)
        fo = torch.empty(pp.image_shape(), dtype=dt, device=dev)

        def fa():
            pp.forward(ft, out=go)
            pp.adjoint(go, out=fo)

        ms = _time_steps(fa, stream, flush, 5, warmup=2)
        inf = pp.info()
        res[name] = {"instance_apps_per_s": len(geoms) * 1000.0 / ms, "ms_per_batch": ms,
                     "samples_per_instance": inf["samples"] // len(geoms),
                     "tile": {k: inf[k] for k in ("m_lanes", "q_piece", "band_rows", "adj_mode", "adj_groups")}}
        del pp, ft, go, fo
        torch.cuda.empty_cache()
    g = geoms[0]
    gr = Geometry(256, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)
    p = wl.params
    f_r = inputs.mixed_phantom(256, p["tubes"], p["gaussians"], seed=p["seeds"][0],
                               width_px=tuple(w * 256 / g.n for w in p["width_px"]))
    d_r = inputs.random_data(gr.n_det, gr.n_t, seed=6)
    outs = {}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        pr = PatPlan(gr, device=dev, image_dtype=dt)
        fw = pr.forward(torch.tensor(f_r, dtype=dt, device=dev))
        ad = pr.adjoint(torch.tensor(d_r, dtype=torch.float32, device=dev))
        torch.cuda.synchronize()
        outs[name] = (fw.double().cpu().numpy(), ad.double().cpu().numpy())
        del pr
    if with_oracle:
        import oracle as O

        O.set_threads(os.cpu_count() or 1)
        og = O.Geometry(gr.n, gr.n_det, gr.arc_start, gr.arc_span, gr.n_t, gr.t_max, gr.n_angles)
        ref_f = O.forward(og, f_r.astype(np.float32).astype(np.float64))
        ref_a = O.adjoint(og, d_r.astype(np.float32).astype(np.float64))
        O.set_threads(1)
        for name, (fw, ad) in outs.items():
            res[name]["rel_l2_fwd_vs_fp64_replica256"] = float(np.linalg.norm(fw - ref_f) / np.linalg.norm(ref_f))
            res[name]["rel_l2_adj_vs_fp64_replica256"] = float(np.linalg.norm(ad - ref_a) / np.linalg.norm(ref_a))
    res["config"] = ("8 x 1024^2 (40 tubes 2-6 px + 10 Gaussians, seeds 5..12), 512 detectors / 270 deg, "
                     "n_t 2048, K 2048; replica 256^2 of seed 5 with the same physical tube widths; adjoint "
                     "error on N(0,1) data")
    return res


# --------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.backends.cudnn.allow_tf32 = False

    from paper_2604_19176_gb300 import PatPlan, inputs

    wl, g, f_true = make_inputs(seed_offset=rank)
    if args.tile:
        vals = [int(x) for x in args.tile.split(",")]
        ml, qp, br, ag, am, sp = vals[:6]
        tc = vals[6] if len(vals) > 6 else 0
        st_ = vals[7] if len(vals) > 7 else 0
        plan = PatPlan(g, device=dev, m_lanes=ml, q_piece=qp, band_rows=br, adj_groups=ag, adj_mode=am,
                       abel_split=sp, tile_cols=tc, adj_jblock=st_)
    else:
        plan = PatPlan(g, device=dev, tune=1)  # autotuned tile shapes (timed at plan creation)
    info = plan.info()
    stream = torch.cuda.current_stream(dev)

    # data: A f_true + 1 % (of max|g|) noise, computed with our forward
    f_t = torch.tensor(f_true, dtype=torch.float32, device=dev)
    g_clean = plan.forward(f_t)
    torch.cuda.synchronize()
    g_meas = torch.tensor(inputs.add_noise(g_clean.double().cpu().numpy(), NOISE, seed=77 + rank),
                          dtype=torch.float32, device=dev)
    # step size from the operator norm (power iteration on A^T A)
    x = torch.rand_like(f_t)
    for _ in range(20):
        x = plan.adjoint(plan.forward(x))
        nrm = float(x.norm())
        x /= nrm
    tau = 1.0 / (nrm + 8.0 * LAM / EPS)

    f_bufs = [torch.zeros_like(f_t), torch.zeros_like(f_t)]
    g_pred = torch.empty_like(g_meas)
    f_adj = torch.empty_like(f_t)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    it = [0]

    def step():
        # one fused projected-gradient TV iteration (pat_tv_step): A f, residual,
        # A^T r, TV gradient and update, ping-ponging the image buffers
        k = it[0]
        plan.tv_step(f_bufs[k & 1], f_bufs[(k + 1) & 1], g_meas, tau, LAM, EPS, nonneg=True)
        it[0] = k + 1

    launches_per_step = 5  # circular means, Abel forward+residual, Abel adjoint, adjoint gather, TV update
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index)
    n_steps = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]

    def load_for(seconds: float):
        # the same flushed steps, untimed, back to back for `seconds` (wall)
        t_end = time.perf_counter() + seconds
        i = 0
        while time.perf_counter() < t_end:
            for _ in range(50):
                flush.fill_(float(i))
                step()
                i += 1
            torch.cuda.synchronize()

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # The timed region lasts a few ms, shorter than the sampling period of
    # nvidia-smi: the clocks are sampled over a window of identical load steps
    # that contains it (CLOCK_WINDOW_S of them before and after).
    if not args.profile:
        clocks.start()
        load_for(CLOCK_WINDOW_S)
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.profiler.start()   # ncu --profile-from-start off: capture the timed steps only
    for i in range(n_steps):
        if not args.profile:
            flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if args.profile:
        torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    if not args.profile:
        load_for(CLOCK_WINDOW_S)
    clk = clocks.stop()
    clk["window"] = (f"nvidia-smi every 20 ms over {CLOCK_WINDOW_S:.1f} s of identical steps, the timed "
                     f"steps, and {CLOCK_WINDOW_S:.1f} s more")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # Per-kernel durations for the roofline: a second pass of the same steps
    # with an event pair around every kernel (the events themselves cost a few
    # microseconds per kernel, so the timed pass above has none).
    plan.set_timing(True)
    for i in range(n_steps):
        flush.fill_(float(i))
        step()
    torch.cuda.synchronize()
    plan.set_timing(False)
    ktimes = plan.kernel_times()
    ms = max_over_ranks(statistics.mean(step_ms), world, dev)
    value = job_value(ms, world)

    # ---- roofline of the dominant kernel --------------------------------
    peaks, peak_kind = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    per_kernel = {k: (v[0] / max(v[1], 1), v[1]) for k, v in ktimes.items() if v[1] > 0}
    total_k = sum(v[0] for v in ktimes.values())
    dom = max(per_kernel, key=lambda k: ktimes[k][0])
    dom_ms = per_kernel[dom][0]
    samples = info["samples"]
    if dom in ("circmean", "adjoint_gather"):
        achieved = samples * BYTES_PER_SAMPLE / (dom_ms * 1e-3) / 1e9
        peak = SMEM_BYTES_PER_CLK_SM * sms * sm_max * 1e6 / 1e9
        roof = {"bound": "alu", "resource": "shared-memory load pipe (4 FP32 texels per bilinear sample)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": load_traffic(dom), "kernel": dom, "kernel_ms": dom_ms,
                "algorithmic": f"{samples} samples x {BYTES_PER_SAMPLE} B per launch",
                "peak_basis": f"{SMEM_BYTES_PER_CLK_SM} B/clk/SM x {sms} SMs x {sm_max:.0f} MHz "
                              f"({peak_kind} sm_max_mhz)"}
    else:
        flops = 2.0 * info["time_macs"]
        achieved = flops / (dom_ms * 1e-3) / 1e12
        peak = 2 * 128 * sms * sm_max * 1e6 / 1e12
        roof = {"bound": "alu", "resource": "FP32 FMA pipe", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": load_traffic(dom), "kernel": dom,
                "kernel_ms": dom_ms}
    roof["kernel_timing"] = ("event pair around every kernel in a second pass of the same steps "
                             "(the timed pass has no per-kernel events)")
    roof["kernel_share"] = {k: round(v[0] / total_k, 4) for k, v in ktimes.items() if v[1] > 0}
    roof["kernel_avg_ms"] = {k: round(v[0], 5) for k, v in per_kernel.items()}

    # ---- end to end through the public API with host buffers ------------
    e2e = None
    if not args.profile:
        h_f = torch.empty(f_t.shape, dtype=torch.float32, pin_memory=True)
        h_f.copy_(f_t.cpu())
        h_g = torch.empty(g_meas.shape, dtype=torch.float32, pin_memory=True)
        h_g.copy_(g_meas.cpu())
        h_out = torch.empty(f_t.shape, dtype=torch.float32, pin_memory=True)
        d_f = torch.empty_like(f_t)
        d_g = torch.empty_like(g_meas)
        d_fo = torch.empty_like(f_t)

        def host_loop(body):
            e_ms = []
            for i in range(min(n_steps, 100) + 3):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                d_f.copy_(h_f, non_blocking=True)
                d_g.copy_(h_g, non_blocking=True)
                h_out.copy_(body(), non_blocking=True)
                b.record(stream)
                b.synchronize()
                if i >= 3:
                    e_ms.append(a.elapsed_time(b))
            return max_over_ranks(statistics.mean(e_ms), world, dev)

        def step_body():
            plan.tv_step(d_f, d_fo, d_g, tau=tau, lam=LAM, eps=EPS)
            return d_fo

        def fwd_adj_body():
            plan.forward(d_f, out=g_pred)
            plan.adjoint(d_g, out=f_adj)
            return f_adj

        em = host_loop(step_body)
        em_sep = host_loop(fwd_adj_body)
        e2e = {"value": job_value(em, world), "unit": UNIT,
               "h2d_bytes_per_step": int(h_f.numel() * 4 + h_g.numel() * 4),
               "d2h_bytes_per_step": int(h_out.numel() * 4), "ms_per_step": em,
               "note": "pinned host f and g copied in, the step timed above (pat_tv_step), the updated image "
                       "copied out, per step",
               "separate_calls": {"value": job_value(em_sep, world), "ms_per_step": em_sep,
                                  "note": "the same copies around pat_forward(f) and pat_adjoint(g) as two calls "
                                          "(no fused time stage)"}}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile:
        cpu = cpu_oracle_timing(g, f_true)

    extras = None
    if rank == 0 and not args.no_extras and not args.profile:
        extras = run_extras(dev, flush, with_oracle=(world == 1))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": n_steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(g),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches_per_step * n_steps,
                "tile_shape": {k: info[k] for k in ("m_lanes", "q_piece", "band_rows", "tile_cols", "bands_max",
                                                    "adj_groups", "adj_mode", "abel_split_fwd", "abel_split_adj",
                                                    "adj_jblock")},
                "samples_per_application": samples, "sample_slots": info["sample_slots"],
                "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms),
                "extras": extras}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()

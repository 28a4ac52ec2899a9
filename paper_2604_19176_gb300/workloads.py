"""Named synthetic workloads: geometry plus the seeded phantom recipe.

The geometries follow the paper's limited-view circular setting (Sec. 2.1:
detectors on an arc of a ring; Sec. 2.4.2: 256 detectors on 270 degrees) at
the sizes this library is measured on.  Phantoms come from
:mod:`paper_2604_19176_gb300.inputs` (Gaussians and vessel tubes standing in
for the paper's datasets, which are not available here).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import inputs
from .api import Geometry


@dataclass(frozen=True)
class Workload:
    name: str
    geometries: tuple
    description: str
    params: dict = field(default_factory=dict)

    def phantoms(self) -> list[np.ndarray]:
        return [make_phantom(g.n, self.params.get("phantom", "vessel"), seed, self.params)
                for g, seed in zip(self.geometries, self.params.get("seeds", range(len(self.geometries))))]


def make_phantom(n: int, kind: str, seed: int, params: dict) -> np.ndarray:
    if kind == "gauss":
        return inputs.gaussian_phantom(n, params.get("count", 5), seed=seed)
    if kind == "vessel":
        return inputs.vessel_phantom(n, params.get("tubes", 12), seed=seed,
                                     width_px=params.get("width_px", (2.0, 4.0)))
    if kind == "mixed":
        return inputs.mixed_phantom(n, params.get("tubes", 12), params.get("gaussians", 5), seed=seed,
                                    width_px=params.get("width_px", (2.0, 4.0)))
    raise ValueError(kind)


def _arc(n, n_det, deg, n_t, K, t_max=2.0):
    return Geometry(n, n_det, 0.0, math.radians(deg), n_t, t_max, K)


def gauss64_full() -> Workload:
    """64x64, 5 Gaussians, 64 detectors on the full circle, 128 times on (0,2], K=128."""
    return Workload("gauss64_full", (_arc(64, 64, 360.0, 128, 128),),
                    "N=64, 5 Gaussians (seed 1), 64 detectors / 360 deg, n_t=128, T=2, K=128",
                    {"phantom": "gauss", "count": 5, "seeds": [1]})


def vessel256_half() -> Workload:
    """256x256 vessel phantom, 128 detectors on 180 degrees, 512 times, K=512."""
    return Workload("vessel256_half", (_arc(256, 128, 180.0, 512, 512),),
                    "N=256, 12 vessel tubes (seed 2), 128 detectors / 180 deg, n_t=512, T=2, K=512",
                    {"phantom": "vessel", "tubes": 12, "seeds": [2], "noise": (0.01, 0.05), "lam": 1e-3,
                     "iters": 500})


def vessel512_half() -> Workload:
    """512x512 variant: 256 detectors on 180 degrees, 1024 times, K=1024."""
    return Workload("vessel512_half", (_arc(512, 256, 180.0, 1024, 1024),),
                    "N=512, 12 vessel tubes (seed 2), 256 detectors / 180 deg, n_t=1024, T=2, K=1024",
                    {"phantom": "vessel", "tubes": 12, "seeds": [2]})


def batch64_uneven(seed: int = 4) -> Workload:
    """64 uneven instances: N, arc, detectors and time samples drawn per instance; K = 2N."""
    rng = np.random.default_rng(seed)
    geoms = []
    for _ in range(64):
        n = int(rng.choice([128, 192, 256, 384]))
        deg = float(rng.choice([90.0, 180.0, 270.0, 360.0]))
        nd = int(rng.choice([64, 128, 256, 512]))
        nt = int(rng.choice([256, 512, 1024]))
        geoms.append(_arc(n, nd, deg, nt, 2 * n))
    return Workload("batch64_uneven", tuple(geoms),
                    "64 instances, N in {128,192,256,384}, arc in {90,180,270,360} deg, "
                    "n_det in {64,128,256,512}, n_t in {256,512,1024}, K=2N (seed 4)",
                    {"phantom": "mixed", "tubes": 12, "gaussians": 5, "seeds": list(range(100, 164))})


def vessel1024_b8() -> Workload:
    """1024x1024, 40 tubes (2-6 px) + 10 Gaussians, 512 detectors on 270 degrees, 2048 times, batch 8."""
    g = _arc(1024, 512, 270.0, 2048, 2048)
    return Workload("vessel1024_b8", (g,) * 8,
                    "N=1024, 40 tubes (2-6 px) + 10 Gaussians, 512 detectors / 270 deg, n_t=2048, K=2048, "
                    "batch 8 (seeds 5..12)",
                    {"phantom": "mixed", "tubes": 40, "gaussians": 10, "width_px": (2.0, 6.0),
                     "seeds": list(range(5, 13))})


def exp760_270() -> Workload:
    """The experimental-data geometry of Sec. 2.4.2: a 760x760 image, 256
    detectors on 270 degrees and 2030 time samples, with a synthetic phantom
    (12 tubes + 5 Gaussians) standing in for the measured one; K = 2N."""
    return Workload("exp760_270", (_arc(760, 256, 270.0, 2030, 1520),),
                    "N=760, 12 vessel tubes + 5 Gaussians (seed 9), 256 detectors / 270 deg, n_t=2030, T=2, K=1520",
                    {"phantom": "mixed", "tubes": 12, "gaussians": 5, "seeds": [9]})


def fine_phantoms(wl: Workload, factor: int = 2) -> list[np.ndarray]:
    """The workload's phantoms rendered on a ``factor`` times finer grid: the
    same analytic objects (tube widths scaled in pixels so that they keep their
    physical width)."""
    params = dict(wl.params)
    if "width_px" in params or params.get("phantom", "vessel") in ("vessel", "mixed"):
        lo, hi = params.get("width_px", (2.0, 4.0))
        params["width_px"] = (lo * factor, hi * factor)
    return [make_phantom(g.n * factor, params.get("phantom", "vessel"), seed, params)
            for g, seed in zip(wl.geometries, params.get("seeds", range(len(wl.geometries))))]


def fine_geometries(wl: Workload, factor: int = 2) -> list[Geometry]:
    """Each geometry on a ``factor`` times finer image grid, with the same
    detectors and time grid (so the same data shape) and factor x K angles."""
    return [Geometry(g.n * factor, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles * factor)
            for g in wl.geometries]


def simulate_fine_data(wl: Workload, factor: int = 2, device=None):
    """Data for the workload's geometries simulated without the inverse crime:
    A applied on a ``factor`` times finer grid to the finely rendered phantoms
    (the paper simulated at 512^2 with a wave solver and reconstructed at 256^2,
    Sec. 2.4.1; here the fine-grid A stands in for the wave solver).  Returns
    the packed FP32 data on ``device``, shaped like a plan of ``wl``'s data."""
    import torch

    from .api import PatPlan

    geoms = fine_geometries(wl, factor)
    plan = PatPlan(geoms, device=device)
    f = torch.tensor(np.concatenate([p.ravel() for p in fine_phantoms(wl, factor)]), dtype=torch.float32,
                     device=plan.device).reshape(plan.image_shape())
    out = plan.forward(f)
    plan.close()
    return out


ALL = {w.__name__: w for w in (gauss64_full, vessel256_half, vessel512_half, batch64_uneven, vessel1024_b8,
                               exp760_270)}

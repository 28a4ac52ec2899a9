"""Python face of the C ABI: a plan object operating on CUDA torch tensors.

PyTorch provides device memory and streams only; every operator step runs in
the library's CUDA kernels (``include/pat.h``).  Shapes:

* single instance: f ``(N, N)``, g ``(n_det, n_t)``;
* B identical instances: f ``(B, N, N)``, g ``(B, n_det, n_t)``;
* uneven instances: flat packed 1-D buffers (see :meth:`PatPlan.layout`).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass
from typing import Iterable, Sequence

import torch

from . import _lib

__all__ = ["Geometry", "PatPlan"]


@dataclass(frozen=True)
class Geometry:
    """One acquisition geometry (the fields of ``pat_geometry_t``)."""

    n: int
    n_det: int
    arc_start: float
    arc_span: float
    n_t: int
    t_max: float
    n_angles: int

    @property
    def n_r(self) -> int:
        return self.n_t + 2

    def to_c(self) -> _lib.PatGeometry:
        return _lib.PatGeometry(self.n, self.n_det, self.arc_start, self.arc_span, self.n_t, self.t_max,
                                self.n_angles)


def _stream_ptr(stream, device) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


class PatPlan:
    """Owner of a ``pat_plan_t`` for a list of geometries on one CUDA device.

    image_dtype: torch.float32 or torch.bfloat16 (storage of f in forward/adjoint).
    Tile options (m_lanes, q_piece, band_rows, tile_cols, adj_groups, ...) map
    to ``pat_options_t``; 0 selects the built-in choice.
    """

    def __init__(self, geoms: Geometry | Sequence[Geometry], *, image_dtype=torch.float32, device=None,
                 m_lanes: int = 0, q_piece: int = 0, band_rows: int = 0, adj_groups: int = 0,
                 adj_mode: int = 0, abel_split: int = 0, tile_cols: int = 0, time_pair: int = 0, schedule: int = 0,
                 tune: int = 0, adj_jblock: int = 0, stream=None):
        self._lib = _lib.load()
        if isinstance(geoms, Geometry):
            geoms = [geoms]
        self.geoms = list(geoms)
        if not self.geoms:
            raise ValueError("at least one geometry is required")
        if image_dtype not in (torch.float32, torch.bfloat16):
            raise ValueError("image_dtype must be torch.float32 or torch.bfloat16")
        self.image_dtype = image_dtype
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
        arr = (_lib.PatGeometry * len(self.geoms))(*[g.to_c() for g in self.geoms])
        opt = _lib.PatOptions()
        opt.image_dtype = 1 if image_dtype == torch.bfloat16 else 0
        opt.schedule = schedule
        opt.tune = tune
        opt.m_lanes, opt.q_piece, opt.band_rows, opt.adj_groups = m_lanes, q_piece, band_rows, adj_groups
        opt.adj_mode = adj_mode
        opt.abel_split = abel_split
        opt.tile_cols = tile_cols
        opt.time_pair = time_pair
        opt.adj_jblock = adj_jblock
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = _stream_ptr(stream, self.device)
            _lib.check("pat_plan_create", self._lib.pat_plan_create(arr, len(self.geoms), ctypes.byref(opt), st,
                                                                    ctypes.byref(handle)))
        self._h = handle
        nb = len(self.geoms) + 1
        fo = (ctypes.c_int64 * nb)()
        go = (ctypes.c_int64 * nb)()
        _lib.check("pat_plan_layout", self._lib.pat_plan_layout(self._h, fo, go))
        self.f_offsets = list(fo)
        self.g_offsets = list(go)
        g0 = self.geoms[0]
        self.uniform = all(g == g0 for g in self.geoms)

    # -- bookkeeping ---------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.check("pat_plan_destroy", self._lib.pat_plan_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def info(self) -> dict:
        inf = _lib.PatPlanInfo()
        _lib.check("pat_plan_info", self._lib.pat_plan_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _lib.PatPlanInfo._fields_ if k != "reserved"}

    def layout(self) -> tuple[list[int], list[int]]:
        return self.f_offsets, self.g_offsets

    @property
    def f_elems(self) -> int:
        return self.f_offsets[-1]

    @property
    def g_elems(self) -> int:
        return self.g_offsets[-1]

    def image_shape(self) -> tuple[int, ...]:
        g = self.geoms[0]
        if not self.uniform:
            return (self.f_elems,)
        return (g.n, g.n) if len(self.geoms) == 1 else (len(self.geoms), g.n, g.n)

    def data_shape(self) -> tuple[int, ...]:
        g = self.geoms[0]
        if not self.uniform:
            return (self.g_elems,)
        return (g.n_det, g.n_t) if len(self.geoms) == 1 else (len(self.geoms), g.n_det, g.n_t)

    def _check(self, t: torch.Tensor, numel: int, dtype, name: str) -> None:
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != self.device.index:
            raise ValueError(f"{name} is on {t.device}, the plan on {self.device}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"{name} must be contiguous with {numel} elements, got {tuple(t.shape)}")

    # -- operators -----------------------------------------------------------
    def forward(self, f: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """g = A f (every instance)."""
        self._check(f, self.f_elems, self.image_dtype, "f")
        if out is None:
            out = torch.empty(self.data_shape(), dtype=torch.float32, device=self.device)
        self._check(out, self.g_elems, torch.float32, "out")
        _lib.check("pat_forward", self._lib.pat_forward(self._h, ctypes.c_void_p(f.data_ptr()),
                                                        ctypes.c_void_p(out.data_ptr()),
                                                        _stream_ptr(stream, self.device)))
        return out

    def adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """f = A^T g (every instance)."""
        self._check(g, self.g_elems, torch.float32, "g")
        if out is None:
            out = torch.empty(self.image_shape(), dtype=self.image_dtype, device=self.device)
        self._check(out, self.f_elems, self.image_dtype, "out")
        _lib.check("pat_adjoint", self._lib.pat_adjoint(self._h, ctypes.c_void_p(g.data_ptr()),
                                                        ctypes.c_void_p(out.data_ptr()),
                                                        _stream_ptr(stream, self.device)))
        return out

    def tv_grad(self, f: torch.Tensor, eps: float, grad: torch.Tensor | None = None, want_value: bool = True,
                stream=None):
        """(TV values per instance, dTV/df) of the smoothed isotropic TV."""
        self._check(f, self.f_elems, torch.float32, "f")
        if grad is None:
            grad = torch.empty_like(f)
        self._check(grad, self.f_elems, torch.float32, "grad")
        val = torch.empty(len(self.geoms), dtype=torch.float32, device=self.device) if want_value else None
        _lib.check("pat_tv_grad", self._lib.pat_tv_grad(
            self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_float(eps), ctypes.c_void_p(grad.data_ptr()),
            ctypes.c_void_p(val.data_ptr() if val is not None else 0), _stream_ptr(stream, self.device)))
        return val, grad

    def tv_value(self, f: torch.Tensor, eps: float, stream=None) -> torch.Tensor:
        self._check(f, self.f_elems, torch.float32, "f")
        val = torch.empty(len(self.geoms), dtype=torch.float32, device=self.device)
        _lib.check("pat_tv_grad", self._lib.pat_tv_grad(
            self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_float(eps), ctypes.c_void_p(0),
            ctypes.c_void_p(val.data_ptr()), _stream_ptr(stream, self.device)))
        return val

    def residual(self, Af: torch.Tensor, g: torch.Tensor, out: torch.Tensor | None = None, scale: float = 1.0,
                 stream=None) -> torch.Tensor:
        """scale * (Af - g)."""
        self._check(Af, self.g_elems, torch.float32, "Af")
        self._check(g, self.g_elems, torch.float32, "g")
        if out is None:
            out = torch.empty_like(Af)
        self._check(out, self.g_elems, torch.float32, "out")
        _lib.check("pat_residual", self._lib.pat_residual(
            self._h, ctypes.c_void_p(Af.data_ptr()), ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_float(scale), _stream_ptr(stream, self.device)))
        return out

    def descent_step(self, f: torch.Tensor, adj: torch.Tensor, tvgrad: torch.Tensor | None, tau: float, lam: float,
                     nonneg: bool = True, delta: torch.Tensor | None = None, stream=None) -> None:
        """In place: f <- [f - tau (adj + lam tvgrad)]_+ ; delta <- (||df||^2, ||f||^2) per instance."""
        self._check(f, self.f_elems, torch.float32, "f")
        self._check(adj, self.f_elems, torch.float32, "adj")
        if tvgrad is not None:
            self._check(tvgrad, self.f_elems, torch.float32, "tvgrad")
        if delta is not None:
            self._check(delta, 2 * len(self.geoms), torch.float32, "delta")
        _lib.check("pat_descent_step", self._lib.pat_descent_step(
            self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(adj.data_ptr()),
            ctypes.c_void_p(tvgrad.data_ptr() if tvgrad is not None else 0), ctypes.c_float(tau),
            ctypes.c_float(lam), 1 if nonneg else 0, ctypes.c_void_p(delta.data_ptr() if delta is not None else 0),
            _stream_ptr(stream, self.device)))

    def tv_step(self, f_in: torch.Tensor, f_out: torch.Tensor, g: torch.Tensor, tau: float, lam: float, eps: float,
                nonneg: bool = True, delta: torch.Tensor | None = None, stream=None) -> None:
        """One projected-gradient TV iteration (Eq. (4)) into f_out (fused kernels)."""
        self._check(f_in, self.f_elems, torch.float32, "f_in")
        self._check(f_out, self.f_elems, torch.float32, "f_out")
        self._check(g, self.g_elems, torch.float32, "g")
        if delta is not None:
            self._check(delta, 2 * len(self.geoms), torch.float32, "delta")
        _lib.check("pat_tv_step", self._lib.pat_tv_step(
            self._h, ctypes.c_void_p(f_in.data_ptr()), ctypes.c_void_p(f_out.data_ptr()),
            ctypes.c_void_p(g.data_ptr()), ctypes.c_float(tau), ctypes.c_float(lam), ctypes.c_float(eps),
            1 if nonneg else 0, ctypes.c_void_p(delta.data_ptr() if delta is not None else 0),
            _stream_ptr(stream, self.device)))

    def pdhg_step(self, f: torch.Tensor, fbar: torch.Tensor, y: torch.Tensor, px: torch.Tensor, py: torch.Tensor,
                  g: torch.Tensor, sigma: float, tau: float, alpha: float, nonneg: bool = True,
                  delta: torch.Tensor | None = None, beta: float = 0.0, mean_target: float = 0.0,
                  fmean: torch.Tensor | None = None, stream=None) -> None:
        """One primal-dual (Chambolle-Pock) TV iteration for Eq. (4), in place on
        f, fbar, y, px, py (and fmean); ``beta`` > 0 adds the mean-intensity
        penalty beta/2 (mean f - mean_target)^2 (see ``pat_pdhg_step``)."""
        for t, name in ((f, "f"), (fbar, "fbar"), (px, "px"), (py, "py")):
            self._check(t, self.f_elems, torch.float32, name)
        self._check(y, self.g_elems, torch.float32, "y")
        self._check(g, self.g_elems, torch.float32, "g")
        if delta is not None:
            self._check(delta, 2 * len(self.geoms), torch.float32, "delta")
        if fmean is not None:
            self._check(fmean, len(self.geoms), torch.float32, "fmean")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)  # noqa: E731
        _lib.check("pat_pdhg_step", self._lib.pat_pdhg_step(
            self._h, ptr(f), ptr(fbar), ptr(y), ptr(px), ptr(py), ptr(g), ctypes.c_float(sigma), ctypes.c_float(tau),
            ctypes.c_float(alpha), 1 if nonneg else 0, ctypes.c_float(beta), ctypes.c_float(mean_target), ptr(fmean),
            ptr(delta), _stream_ptr(stream, self.device)))

    def set_timing(self, enable: bool) -> None:
        """Bracket every kernel launch of this plan with CUDA events."""
        _lib.check("pat_plan_set_timing", self._lib.pat_plan_set_timing(self._h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """{kernel kind: (total ms, launches)} since the last call (synchronises)."""
        n = len(_lib.KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _lib.check("pat_plan_kernel_times", self._lib.pat_plan_kernel_times(self._h, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(_lib.KERNEL_KINDS)}

    def sync_status(self, stream=None) -> int:
        return int(self._lib.pat_plan_sync_status(self._h, _stream_ptr(stream, self.device)))

    def set_wait_probe(self, clocks: int) -> None:
        """Test hook: the next circular-mean launch has one CTA wait on a barrier
        nothing completes, bounded by ``clocks`` SM cycles (see pat_plan_set_wait_probe)."""
        _lib.check("pat_plan_set_wait_probe", self._lib.pat_plan_set_wait_probe(self._h, int(clocks)))

    def set_bounds_probe(self, enable: bool = True) -> None:
        """Test hook of debug builds: the next list gather plants one out-of-range
        detector index for its bounds check to report (see pat_plan_set_bounds_probe)."""
        _lib.check("pat_plan_set_bounds_probe", self._lib.pat_plan_set_bounds_probe(self._h, 1 if enable else 0))


def geometry_from(obj) -> Geometry:
    """Geometry from any object with the same fields (e.g. a dict)."""
    if isinstance(obj, Geometry):
        return obj
    if isinstance(obj, dict):
        return Geometry(**obj)
    return Geometry(obj.n, obj.n_det, obj.arc_start, obj.arc_span, obj.n_t, obj.t_max, obj.n_angles)


def full_circle(n: int, n_det: int, n_t: int, n_angles: int, t_max: float = 2.0) -> Geometry:
    return Geometry(n, n_det, 0.0, 2.0 * math.pi, n_t, t_max, n_angles)


def arc(n: int, n_det: int, degrees: float, n_t: int, n_angles: int, t_max: float = 2.0,
        start_degrees: float = 0.0) -> Geometry:
    return Geometry(n, n_det, math.radians(start_degrees), math.radians(degrees), n_t, t_max, n_angles)


def geometries(items: Iterable) -> list[Geometry]:
    return [geometry_from(x) for x in items]

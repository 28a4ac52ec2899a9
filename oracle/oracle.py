"""ctypes binding of the plain-C FP64 oracle (``pat_oracle.c``).

Test infrastructure only: the product library neither imports nor links this
module.  Every function mirrors one C entry point; the C source carries the
derivations (2D Poisson formula for Eq. (1)-(2), operator equation Eq. (3),
TV term of Eq. (4)-(5)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pat_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

__all__ = [
    "Geometry", "build", "load", "set_threads", "get_threads", "abel_matrix",
    "abel_weights", "bilinear", "circle_mean", "detectors", "circular_means",
    "forward", "adjoint_time", "adjoint_means", "adjoint", "count_samples", "tv",
]


@dataclass(frozen=True)
class Geometry:
    """Acquisition geometry (see ``pat_oracle.h``).

    n: image side N (pixels on [-1,1]^2); n_det detectors on the arc that
    starts at ``arc_start`` and spans ``arc_span`` radians; n_t time samples
    on (0, t_max]; n_angles angular nodes K per circular mean.
    """

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


class _CGeom(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("n_det", ctypes.c_int), ("arc_start", ctypes.c_double),
        ("arc_span", ctypes.c_double), ("n_t", ctypes.c_int), ("t_max", ctypes.c_double),
        ("n_angles", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile ``pat_oracle.c`` into ``liboracle.so`` with the host gcc."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pat_oracle.h"))
    ):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    gp = ctypes.POINTER(_CGeom)
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    lib.orc_get_threads.restype = ctypes.c_int
    lib.orc_abel_matrix.argtypes = [ctypes.c_int, dp]
    lib.orc_abel_weights.argtypes = [ctypes.c_double, ctypes.c_int, dp]
    lib.orc_bilinear.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    lib.orc_bilinear.restype = ctypes.c_double
    lib.orc_circle_mean.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.orc_circle_mean.restype = ctypes.c_double
    lib.orc_detectors.argtypes = [gp, dp]
    lib.orc_circular_means.argtypes = [gp, dp, dp]
    lib.orc_forward.argtypes = [gp, dp, dp]
    lib.orc_adjoint_time.argtypes = [gp, dp, dp]
    lib.orc_adjoint_means.argtypes = [gp, dp, dp]
    lib.orc_adjoint.argtypes = [gp, dp, dp]
    lib.orc_count_samples.argtypes = [gp]
    lib.orc_count_samples.restype = ctypes.c_longlong
    lib.orc_tv.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
    lib.orc_tv.restype = ctypes.c_double
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _in(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _cg(g: Geometry) -> _CGeom:
    return _CGeom(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


def set_threads(n: int) -> None:
    load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(load().orc_get_threads())


def abel_matrix(n_t: int) -> np.ndarray:
    """P, shape (n_t, n_t + 2): g[j, k-1] = sum_m P[k-1, m] M[j, m]."""
    P = np.zeros((n_t, n_t + 2))
    load().orc_abel_matrix(n_t, _ptr(P))
    return P


def abel_weights(tau: float, n_r: int) -> np.ndarray:
    w = np.zeros(n_r)
    load().orc_abel_weights(float(tau), int(n_r), _ptr(w))
    return w


def bilinear(f: np.ndarray, sx: float, sy: float) -> float:
    f = _in(f)
    return float(load().orc_bilinear(_ptr(f), f.shape[0], float(sx), float(sy)))


def circle_mean(f: np.ndarray, cx: float, cy: float, r: float, K: int) -> float:
    f = _in(f)
    return float(load().orc_circle_mean(_ptr(f), f.shape[0], float(cx), float(cy), float(r), int(K)))


def detectors(g: Geometry) -> np.ndarray:
    xy = np.zeros((g.n_det, 2))
    cg = _cg(g)
    load().orc_detectors(ctypes.byref(cg), _ptr(xy))
    return xy


def circular_means(g: Geometry, f: np.ndarray) -> np.ndarray:
    f = _in(f, (g.n, g.n))
    M = np.zeros((g.n_det, g.n_r))
    cg = _cg(g)
    load().orc_circular_means(ctypes.byref(cg), _ptr(f), _ptr(M))
    return M


def forward(g: Geometry, f: np.ndarray) -> np.ndarray:
    """g = A f, shape (n_det, n_t)."""
    f = _in(f, (g.n, g.n))
    out = np.zeros((g.n_det, g.n_t))
    cg = _cg(g)
    load().orc_forward(ctypes.byref(cg), _ptr(f), _ptr(out))
    return out


def adjoint_time(g: Geometry, gbar: np.ndarray) -> np.ndarray:
    gbar = _in(gbar, (g.n_det, g.n_t))
    Mbar = np.zeros((g.n_det, g.n_r))
    cg = _cg(g)
    load().orc_adjoint_time(ctypes.byref(cg), _ptr(gbar), _ptr(Mbar))
    return Mbar


def adjoint_means(g: Geometry, Mbar: np.ndarray) -> np.ndarray:
    Mbar = _in(Mbar, (g.n_det, g.n_r))
    fbar = np.zeros((g.n, g.n))
    cg = _cg(g)
    load().orc_adjoint_means(ctypes.byref(cg), _ptr(Mbar), _ptr(fbar))
    return fbar


def adjoint(g: Geometry, gbar: np.ndarray) -> np.ndarray:
    """f = A^T gbar, shape (N, N)."""
    gbar = _in(gbar, (g.n_det, g.n_t))
    fbar = np.zeros((g.n, g.n))
    cg = _cg(g)
    load().orc_adjoint(ctypes.byref(cg), _ptr(gbar), _ptr(fbar))
    return fbar


def count_samples(g: Geometry) -> int:
    cg = _cg(g)
    return int(load().orc_count_samples(ctypes.byref(cg)))


def tv(f: np.ndarray, eps: float, with_grad: bool = True):
    """Smoothed isotropic TV value (and gradient) of an N x N image."""
    f = _in(f)
    n = f.shape[0]
    grad = np.zeros((n, n)) if with_grad else None
    val = load().orc_tv(n, float(eps), _ptr(f), _ptr(grad) if with_grad else None)
    return (float(val), grad) if with_grad else float(val)

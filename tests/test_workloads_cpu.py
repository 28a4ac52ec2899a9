"""CPU checks of the synthetic workloads: the fine-grid rendering used for data
without the inverse crime keeps the phantom's physical size, and the named
geometries are the ones the paper describes (Sec. 2.4.2: 256 detectors on 270
degrees, 2030 time samples, 760 x 760 images)."""
import math

import numpy as np

from paper_2604_19176_gb300 import workloads


def _block_mean(a, k):
    n = a.shape[0] // k
    return a.reshape(n, k, n, k).mean(axis=(1, 3))


def test_fine_phantom_keeps_physical_width():
    """2x2 block means of the 2x finer rendering reproduce the coarse phantom
    (same tubes, same physical widths); rendering the fine grid with unscaled
    pixel widths (tubes half as wide) would not."""
    wl = workloads.Workload("t", (workloads._arc(64, 16, 180.0, 32, 32),), "t",
                            {"phantom": "vessel", "tubes": 6, "seeds": [3]})
    coarse = wl.phantoms()[0]
    fine = workloads.fine_phantoms(wl, 2)[0]
    assert fine.shape == (128, 128)
    err = np.linalg.norm(_block_mean(fine, 2) - coarse) / np.linalg.norm(coarse)
    thin = workloads.make_phantom(128, "vessel", 3, {"tubes": 6})
    err_thin = np.linalg.norm(_block_mean(thin, 2) - coarse) / np.linalg.norm(coarse)
    assert err < 0.2 and err_thin > 2 * err


def test_fine_geometry_keeps_detectors_and_time_grid():
    wl = workloads.vessel256_half()
    (fg,) = workloads.fine_geometries(wl, 2)
    (g,) = wl.geometries
    assert (fg.n, fg.n_angles) == (2 * g.n, 2 * g.n_angles)
    assert (fg.n_det, fg.arc_start, fg.arc_span, fg.n_t, fg.t_max) == (g.n_det, g.arc_start, g.arc_span, g.n_t,
                                                                        g.t_max)


def test_experimental_geometry():
    (g,) = workloads.exp760_270().geometries
    assert (g.n, g.n_det, g.n_t) == (760, 256, 2030)
    assert abs(math.degrees(g.arc_span) - 270.0) < 1e-12

"""The debug build (-DPAT_DEBUG): device-side bounds checks that report, not trap.

The library is rebuilt with the checks (build.build(debug=True)) and driven in
a child process, since this process already holds the release build.  The
child checks that
  - every list form (run-pair codes, one-sample codes, fraction lists) and the
    fused TV step run clean: results match the FP64 oracle and the status word
    stays clear (the checks raise no false alarm);
  - a planted out-of-range detector index (pat_plan_set_bounds_probe) is
    reported once by pat_plan_sync_status as PAT_ERR_BOUNDS, with the kernel
    carrying on, and the next calls are correct again.
The planted index addresses only memory inside the plan's own allocations, so
the run cannot fault even if a check were missing.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r"""
    import math, sys
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2604_19176_gb300 import _lib, build
    lib = _lib.load(build.build(debug=True))       # before any plan: the operators use this build
    assert lib.pat_debug_build() == 1
    import torch
    import oracle as O
    from paper_2604_19176_gb300 import Geometry, PatPlan, inputs

    PAT_OK, PAT_ERR_BOUNDS = 0, 7
    dev = torch.device("cuda", 0)

    def og(g):
        return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)

    def rel(a, b):
        return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))

    g = Geometry(96, 24, 0.3, 1.2 * math.pi, 64, 2.0, 96)
    f_np = inputs.random_image(96, seed=51).astype(np.float32)
    d_np = inputs.random_data(24, 64, seed=52).astype(np.float32)
    f = torch.tensor(f_np, device=dev)
    d = torch.tensor(d_np, device=dev)
    ref_g = O.forward(og(g), f_np.astype(np.float64))
    ref_f = O.adjoint(og(g), d_np.astype(np.float64))

    for mode in (4, 1, 3):   # run-pair code lists, one-sample code lists, fraction lists
        plan = PatPlan(g, device=dev, adj_mode=mode)
        assert plan.info()["adj_mode"] == mode, (mode, plan.info()["adj_mode"])
        out_g = plan.forward(f).double().cpu().numpy()
        out_f = plan.adjoint(d).double().cpu().numpy()
        assert plan.sync_status() == PAT_OK, mode
        assert rel(out_g, ref_g) <= 1e-5 and rel(out_f, ref_f) <= 1e-5, (mode, rel(out_g, ref_g), rel(out_f, ref_f))

        plan.set_bounds_probe()
        plan.adjoint(d)                             # one entry is skipped: this result is undefined
        assert plan.sync_status() == PAT_ERR_BOUNDS, mode
        assert plan.sync_status() == PAT_OK, mode   # reported once, then cleared
        out_f = plan.adjoint(d).double().cpu().numpy()   # the probe disarmed itself
        assert plan.sync_status() == PAT_OK, mode
        assert rel(out_f, ref_f) <= 1e-5, (mode, rel(out_f, ref_f))
        print("mode", mode, "ok", flush=True)

    # the fused TV step (circular means, fused time stage, gather, TV update)
    plan = PatPlan(g, device=dev)
    f0 = torch.zeros_like(f)
    f1 = torch.empty_like(f)
    gmeas = torch.tensor(ref_g.astype(np.float32), device=dev)
    plan.tv_step(f0 + 0.1, f1, gmeas, tau=0.01, lam=1e-3, eps=1e-3)
    torch.cuda.synchronize()
    assert plan.sync_status() == PAT_OK
    assert bool(torch.isfinite(f1).all())
    plan.set_bounds_probe()
    plan.tv_step(f0 + 0.1, f1, gmeas, tau=0.01, lam=1e-3, eps=1e-3)
    assert plan.sync_status() == PAT_ERR_BOUNDS
    print("tv_step ok", flush=True)
""")


def test_debug_build_checks_report_without_trapping():
    code = "ROOT = " + repr(ROOT) + "\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "tv_step ok" in r.stdout

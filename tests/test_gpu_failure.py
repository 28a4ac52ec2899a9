"""The failure path of the bounded device-side waits, exercised without a fault.

pat_plan_set_wait_probe makes one CTA of the next circular-mean launch wait,
with a short bound (1e5 SM clocks, about 50 us), on an mbarrier that nothing
completes.  The wait runs out, records PAT_ERR_TIMEOUT in the plan's device
status word and the CTA returns early, so that call's result is incomplete.
The tests check that the next calls are correct (against the FP64 oracle and
against the same calls on an untouched plan) and that pat_plan_sync_status
reports the timeout once.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_19176_gb300 import Geometry, PatPlan, inputs

pytestmark = pytest.mark.gpu

PAT_OK, PAT_ERR_TIMEOUT = 0, 5
PROBE_CLOCKS = 100_000


def og(g):
    return O.Geometry(g.n, g.n_det, g.arc_start, g.arc_span, g.n_t, g.t_max, g.n_angles)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_wait_probe_times_out_and_sync_status_recovers(cuda_dev):
    g = Geometry(96, 24, 0.3, 1.2 * math.pi, 64, 2.0, 96)
    plan = PatPlan(g, device=cuda_dev)
    f_np = inputs.random_image(96, seed=31).astype(np.float32)
    d_np = inputs.random_data(24, 64, seed=32).astype(np.float32)
    f = torch.tensor(f_np, device=cuda_dev)
    d = torch.tensor(d_np, device=cuda_dev)
    ref_g = O.forward(og(g), f_np.astype(np.float64))
    ref_f = O.adjoint(og(g), d_np.astype(np.float64))

    assert plan.sync_status() == PAT_OK
    plan.set_wait_probe(PROBE_CLOCKS)
    plan.forward(f)                              # one CTA gives up; this result is undefined
    torch.cuda.synchronize()
    # the next calls are correct before the status is read (no state is left armed)
    out_g = plan.forward(f).double().cpu().numpy()
    assert rel(out_g, ref_g) <= 1e-5
    assert plan.sync_status() == PAT_ERR_TIMEOUT
    assert plan.sync_status() == PAT_OK          # reported once, then cleared
    # the probe disarmed itself after one launch
    for _ in range(2):
        out_g = plan.forward(f).double().cpu().numpy()
        out_f = plan.adjoint(d).double().cpu().numpy()
        assert plan.sync_status() == PAT_OK
        assert rel(out_g, ref_g) <= 1e-5
        assert rel(out_f, ref_f) <= 1e-5


def test_wait_probe_in_the_fused_tv_step(cuda_dev):
    g = Geometry(64, 16, 0.0, math.pi, 48, 2.0, 64)
    plan = PatPlan(g, device=cuda_dev)
    fresh = PatPlan(g, device=cuda_dev)
    f0 = torch.tensor(np.abs(inputs.random_image(64, seed=33)), dtype=torch.float32, device=cuda_dev)
    data = torch.tensor(inputs.random_data(16, 48, seed=34), dtype=torch.float32, device=cuda_dev)
    out = torch.empty_like(f0)
    plan.set_wait_probe(PROBE_CLOCKS)
    plan.tv_step(f0, out, data, 0.05, 0.1, 1e-2)
    torch.cuda.synchronize()
    assert plan.sync_status() == PAT_ERR_TIMEOUT
    assert plan.sync_status() == PAT_OK
    a, b = torch.empty_like(f0), torch.empty_like(f0)
    plan.tv_step(f0, a, data, 0.05, 0.1, 1e-2)
    fresh.tv_step(f0, b, data, 0.05, 0.1, 1e-2)
    torch.cuda.synchronize()
    assert plan.sync_status() == PAT_OK
    assert torch.equal(a, b)


def test_wait_probe_argument_checks(cuda_dev):
    from paper_2604_19176_gb300._lib import PatError
    plan = PatPlan(Geometry(32, 8, 0.0, math.pi, 16, 2.0, 16), device=cuda_dev)
    with pytest.raises(PatError):
        plan.set_wait_probe(-1)
    plan.set_wait_probe(0)                       # disarm: a no-op here
    plan.forward(torch.zeros(32, 32, device=cuda_dev))
    assert plan.sync_status() == PAT_OK


def test_forced_allocation_failures_free_everything(cuda_dev):
    """pat_debug_fail_alloc makes the k-th device allocation of the next plan
    creation fail: every k up to the number of allocations returns
    PAT_ERR_OOM with nothing left allocated, and past it the plan is built
    and correct (host-side injection: nothing runs out on the GPU)."""
    from paper_2604_19176_gb300 import _lib

    lib = _lib.load()
    g = Geometry(64, 16, 0.1, math.pi, 48, 2.0, 64)
    f_np = inputs.random_image(64, seed=61).astype(np.float32)
    ref_g = O.forward(og(g), f_np.astype(np.float64))
    PatPlan(g, device=cuda_dev).close()   # first creation loads the kernels plan creation uses
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for k in range(16):
            assert lib.pat_debug_fail_alloc(k) == 0
            try:
                plan = PatPlan(g, device=cuda_dev)
            except _lib.PatError as e:
                assert e.status == 3, e.status             # PAT_ERR_OOM
                torch.cuda.synchronize()
                assert free0 - torch.cuda.mem_get_info()[0] < (1 << 20), k   # nothing leaked
                failed += 1
                continue
            lib.pat_debug_fail_alloc(-1)                    # k was past the last allocation
            out = plan.forward(torch.tensor(f_np, device=cuda_dev)).double().cpu().numpy()
            assert plan.sync_status() == PAT_OK
            assert rel(out, ref_g) <= 1e-5
            plan.close()
            break
        else:
            raise AssertionError("plan creation kept failing")
    finally:
        lib.pat_debug_fail_alloc(-1)
    assert failed >= 3   # tables, workspace and the adjoint lists at least

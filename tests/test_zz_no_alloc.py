"""pat_tv_grad_noalloc: the TV value and gradient for callers that cannot allocate.

Callers running under another framework's allocator, in a real-time loop that
must not call cudaMalloc, or anywhere allocation is forbidden cannot create a
plan (plans allocate).  This entry point serves them from a fixed static
scratch array.  The test calls it through the C ABI and checks it against the
plan-based pat_tv_grad on two calls in a row (the second with new data, so
stale scratch contents from the first call would show), plus the size limit.
The file is named to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2604_19176_gb300 import Geometry, PatPlan, _lib, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def test_noalloc_tv_matches_plan_tv_on_two_calls(cuda_dev):
    lib = _lib.load()
    n, batch, eps = 96, 3, 1e-2
    plan = PatPlan([Geometry(n, 8, 0.0, math.pi, 16, 2.0, 16)] * batch, device=cuda_dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(cuda_dev).cuda_stream)
    for call in range(2):
        imgs = np.stack([inputs.vessel_phantom(n, 6, seed=40 + 10 * call + b) + 0.05 * inputs.random_image(n, seed=b)
                         for b in range(batch)])
        f = torch.tensor(imgs, dtype=torch.float32, device=cuda_dev)
        ref_val, ref_grad = plan.tv_grad(f, eps)
        grad = torch.full_like(f, float("nan"))
        val = torch.full((batch,), float("nan"), dtype=torch.float32, device=cuda_dev)
        status = lib.pat_tv_grad_noalloc(_ptr(f), n, batch, ctypes.c_float(eps), _ptr(grad), _ptr(val), stream)
        assert status == 0, _lib.STATUS_NAMES.get(status)
        torch.cuda.synchronize()
        assert torch.all(torch.isfinite(val)) and torch.all(torch.isfinite(grad))
        rv = (val.double() - ref_val.double()).abs() / ref_val.double().abs()
        assert float(rv.max()) <= TOL
        rg = (grad.double() - ref_grad.double()).norm() / ref_grad.double().norm()
        assert float(rg) <= TOL
        # value only (no gradient buffer)
        val2 = torch.zeros_like(val)
        assert lib.pat_tv_grad_noalloc(_ptr(f), n, batch, ctypes.c_float(eps), _ptr(None), _ptr(val2), stream) == 0
        torch.cuda.synchronize()
        assert float(((val2.double() - ref_val.double()).abs() / ref_val.double().abs()).max()) <= TOL


def test_noalloc_tv_rejects_batches_beyond_the_scratch(cuda_dev):
    lib = _lib.load()
    f = torch.zeros(16, device=cuda_dev)
    val = torch.zeros(4, device=cuda_dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(cuda_dev).cuda_stream)
    # 4096 x 4096 needs 128 x 512 = 65536 tiles per image: two images exceed the scratch
    status = lib.pat_tv_grad_noalloc(_ptr(f), 4096, 2, ctypes.c_float(1e-3), _ptr(None), _ptr(val), stream)
    assert status == 1  # PAT_ERR_INVALID_ARG, nothing enqueued
    assert lib.pat_tv_grad_noalloc(_ptr(f), 0, 1, ctypes.c_float(1e-3), _ptr(None), _ptr(val), stream) == 1

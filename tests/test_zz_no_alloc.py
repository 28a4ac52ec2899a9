"""pat_tv_grad_noalloc: the TV value and gradient for callers that cannot allocate.

Callers running under another framework's allocator, in a real-time loop that
must not call cudaMalloc, or anywhere allocation is forbidden cannot create a
plan (plans allocate).  This entry point serves them from a fixed static
scratch array.  The tests call it through the C ABI and check it against the
plan-based pat_tv_grad and the FP64 oracle on two calls in a row (the second
with new data and a smaller batch, so stale scratch contents from the first
call would show), on image sides that leave partial 32 x 8 tiles, on a
gradient-only call larger than the scratch, and check the refusals (size
limit, a gradient or value buffer overlapping the images).  The file is named
to be collected last.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2604_19176_gb300 import Geometry, PatPlan, _lib, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _ptr(t, offset_elems=0):
    return ctypes.c_void_p(t.data_ptr() + 4 * offset_elems if t is not None else 0)


def _images(n, batch, seed):
    return np.stack([inputs.vessel_phantom(n, 6, seed=seed + b) + 0.05 * inputs.random_image(n, seed=seed + 100 + b)
                     for b in range(batch)]).astype(np.float32)


@pytest.mark.parametrize("n", [96, 100, 37])
def test_noalloc_tv_matches_plan_and_oracle_on_two_calls(cuda_dev, n):
    lib = _lib.load()
    eps = 1e-2
    stream = ctypes.c_void_p(torch.cuda.current_stream(cuda_dev).cuda_stream)
    for call, batch in enumerate((3, 2)):      # the second call is smaller: stale scratch would show
        imgs = _images(n, batch, 40 + 10 * call)
        f = torch.tensor(imgs, device=cuda_dev)
        grad = torch.full_like(f, float("nan"))
        val = torch.full((batch,), float("nan"), dtype=torch.float32, device=cuda_dev)
        status = lib.pat_tv_grad_noalloc(_ptr(f), n, batch, ctypes.c_float(eps), _ptr(grad), _ptr(val), stream)
        assert status == 0, _lib.STATUS_NAMES.get(status)
        torch.cuda.synchronize()
        assert torch.all(torch.isfinite(val)) and torch.all(torch.isfinite(grad))
        if n % 4 == 0:   # plans take N a multiple of 4
            plan = PatPlan([Geometry(n, 8, 0.0, math.pi, 16, 2.0, 16)] * batch, device=cuda_dev)
            ref_val, ref_grad = plan.tv_grad(f, eps)
            torch.cuda.synchronize()
            assert float(((val.double() - ref_val.double()).abs() / ref_val.double().abs()).max()) <= TOL
            assert float((grad.double() - ref_grad.double()).norm() / ref_grad.double().norm()) <= TOL
            plan.close()
        for b in range(batch):
            rv, rg = O.tv(imgs[b].astype(np.float64), eps)
            assert abs(float(val[b]) - rv) <= TOL * rv
            g = grad[b].double().cpu().numpy()
            assert np.linalg.norm(g - rg) <= TOL * np.linalg.norm(rg)
        # value only (no gradient buffer)
        val2 = torch.zeros_like(val)
        assert lib.pat_tv_grad_noalloc(_ptr(f), n, batch, ctypes.c_float(eps), _ptr(None), _ptr(val2), stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(val2, val)


def test_noalloc_gradient_only_beyond_the_scratch(cuda_dev):
    """A gradient needs no scratch: 2 images of 2048^2 (twice the value's tile
    limit) are accepted without a value buffer and match the oracle."""
    lib = _lib.load()
    n, batch, eps = 2048, 2, 1e-2
    stream = ctypes.c_void_p(torch.cuda.current_stream(cuda_dev).cuda_stream)
    imgs = np.stack([inputs.random_image(n, seed=70 + b) for b in range(batch)]).astype(np.float32)
    f = torch.tensor(imgs, device=cuda_dev)
    grad = torch.full_like(f, float("nan"))
    val = torch.zeros(batch, device=cuda_dev)
    # with a value buffer the tiles exceed the scratch: refused, nothing enqueued
    assert lib.pat_tv_grad_noalloc(_ptr(f), n, 8, ctypes.c_float(eps), _ptr(None), _ptr(val), stream) == 1
    assert lib.pat_tv_grad_noalloc(_ptr(f), n, batch, ctypes.c_float(eps), _ptr(grad), _ptr(None), stream) == 0
    torch.cuda.synchronize()
    for b in range(batch):
        _, rg = O.tv(imgs[b].astype(np.float64), eps)
        g = grad[b].double().cpu().numpy()
        assert np.linalg.norm(g - rg) <= TOL * np.linalg.norm(rg)


def test_noalloc_tv_refusals(cuda_dev):
    lib = _lib.load()
    n = 64
    f = torch.zeros(2, n, n, device=cuda_dev)
    g = torch.zeros(2, n, n, device=cuda_dev)
    val = torch.zeros(4, device=cuda_dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(cuda_dev).cuda_stream)
    e = ctypes.c_float(1e-3)
    # 4096 x 4096 needs 128 x 512 = 65536 tiles per image: two images exceed the scratch
    assert lib.pat_tv_grad_noalloc(_ptr(f), 4096, 2, e, _ptr(None), _ptr(val), stream) == 1
    assert lib.pat_tv_grad_noalloc(_ptr(f), 0, 1, e, _ptr(None), _ptr(val), stream) == 1
    # in place, or a gradient overlapping the images by one row: refused
    assert lib.pat_tv_grad_noalloc(_ptr(f), n, 2, e, _ptr(f), _ptr(None), stream) == 1
    assert lib.pat_tv_grad_noalloc(_ptr(f), n, 2, e, _ptr(f, n), _ptr(None), stream) == 1
    # a value buffer inside the images or inside the gradient: refused
    assert lib.pat_tv_grad_noalloc(_ptr(f), n, 2, e, _ptr(g), _ptr(f, 5), stream) == 1
    assert lib.pat_tv_grad_noalloc(_ptr(f), n, 2, e, _ptr(g), _ptr(g, 7), stream) == 1
    # disjoint buffers are accepted
    assert lib.pat_tv_grad_noalloc(_ptr(f), n, 2, e, _ptr(g), _ptr(val), stream) == 0
    torch.cuda.synchronize()

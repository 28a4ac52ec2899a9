"""CPU-only checks of the C ABI: the library builds and loads, exports every
symbol include/pat.h declares, and validates arguments on the host before
touching the GPU (no compute call is made here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "pat.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:pat_status_t|const char\*|int32_t)\s+(pat_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2604_19176_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_header_declares_the_expected_calls():
    syms = declared_symbols()
    from paper_2604_19176_gb300._lib import EXPORTED

    assert set(syms) == set(EXPORTED)
    for core in ("pat_plan_create", "pat_forward", "pat_adjoint", "pat_tv_grad", "pat_plan_destroy"):
        assert core in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.pat_status_string(0) == b"PAT_OK"
    assert lib.pat_status_string(6) == b"PAT_ERR_BAD_PLAN"
    assert lib.pat_status_string(7) == b"PAT_ERR_BOUNDS"
    # the allocation-failure hook is host state only: arming and disarming needs no GPU
    assert lib.pat_debug_fail_alloc(3) == 0
    assert lib.pat_debug_fail_alloc(-1) == 0
    assert lib.pat_status_string(99) == b"PAT_ERR_UNKNOWN"


def test_release_and_debug_builds(lib):
    """The release library has no debug checks; the -DPAT_DEBUG build loads
    (no GPU needed), exports the same symbols and says it is a debug build."""
    from paper_2604_19176_gb300 import _lib, build

    assert lib.pat_debug_build() == 0
    assert lib.pat_plan_set_bounds_probe(None, 1) == 6
    dbg = _lib.open_library(build.build(debug=True))
    for name in declared_symbols():
        assert hasattr(dbg, name), name
    assert dbg.pat_debug_build() == 1
    assert dbg.pat_plan_set_bounds_probe(None, 1) == 6
    assert dbg.pat_forward(None, None, None, None) == 6


def test_host_validation_without_gpu(lib):
    from paper_2604_19176_gb300 import _lib

    h = ctypes.c_void_p()
    geom = _lib.PatGeometry(64, 8, 0.0, 3.14, 16, 2.0, 16)
    assert lib.pat_plan_create(None, 1, None, None, ctypes.byref(h)) == 1
    assert lib.pat_plan_create(ctypes.byref(geom), 0, None, None, ctypes.byref(h)) == 1
    assert lib.pat_plan_create(ctypes.byref(geom), 1, None, None, None) == 1
    bad = _lib.PatGeometry(64, 8, 0.0, 3.14, 16, -1.0, 16)
    assert lib.pat_plan_create(ctypes.byref(bad), 1, None, None, ctypes.byref(h)) == 1
    opt = _lib.PatOptions()
    opt.m_lanes = 5
    assert lib.pat_plan_create(ctypes.byref(geom), 1, ctypes.byref(opt), None, ctypes.byref(h)) == 1
    for field, value in (("adj_mode", 5), ("adj_mode", -1), ("adj_jblock", -1), ("adj_jblock", 16385)):
        opt = _lib.PatOptions()
        setattr(opt, field, value)
        assert lib.pat_plan_create(ctypes.byref(geom), 1, ctypes.byref(opt), None, ctypes.byref(h)) == 1
    # calls on a handle that is not a live plan
    assert lib.pat_forward(None, None, None, None) == 6
    assert lib.pat_adjoint(ctypes.c_void_p(12345), None, None, None) == 6
    assert lib.pat_tv_grad(None, None, ctypes.c_float(1e-3), None, None, None) == 6
    assert lib.pat_plan_destroy(None) == 6
    assert lib.pat_plan_info(None, None) == 6
    f = ctypes.c_float
    assert lib.pat_pdhg_step(None, None, None, None, None, None, None, f(0.1), f(0.1), f(1e-3), 1, f(0.0), f(0.0),
                             None, None, None) == 6
    assert lib.pat_tv_step(None, None, None, None, f(0.1), f(1e-3), f(1e-3), 1, None, None) == 6

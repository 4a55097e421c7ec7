"""The C-ABI library builds, loads and exports every function include/ashrt.h
declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ashrt.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def cdll():
    from paper_1711_10214_gb300 import ashrt, build
    if not os.path.exists(ashrt.LIB_PATH):
        build.build()
    return ashrt.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("ashrt_plan_create", "ashrt_forward", "ashrt_adjoint", "robust_irls_deblend",
              "ashrt_plan_destroy", "ashrt_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(cdll):
    for name in _declared_functions():
        assert hasattr(cdll, name), name


def test_host_side_calls_without_gpu(cdll):
    from paper_1711_10214_gb300 import ashrt
    o = ashrt.AshrtOpts()
    cdll.ashrt_default_opts(ctypes.byref(o))
    assert (o.pad_t, o.pad_x, o.max_batch, o.with_solver) == (2, 2, 1, 0)
    io = ashrt.IrlsOpts()
    cdll.irls_default_opts(ctypes.byref(io))
    assert (io.p, io.q, io.n_outer, io.n_cg, io.b_r) == (1.0, 1.0, 5, 20, 1.345)
    assert cdll.ashrt_status_string(4) == b"ASHRT_ENAN"
    # argument errors are reported before any CUDA call
    h = ctypes.c_void_p()
    v = (ctypes.c_float * 1)(1500.0)
    st = cdll.ashrt_plan_create(ctypes.byref(h), 1, 64, 0.004, 12.5, v, 1, None, 0, None, 1, None)
    assert st == 1 and h.value is None
    assert b"nt >= 2" in cdll.ashrt_last_error()
    ax = (ctypes.c_float * 3)(0.0, 12.5, 30.0)     # apex grid must equal the trace grid
    st = cdll.ashrt_plan_create(ctypes.byref(h), 64, 3, 0.004, 12.5, v, 1, ax, 3, None, 1, None)
    assert st == 1 and b"x_a must equal x" in cdll.ashrt_last_error()


def test_time_domain_argument_checks_without_gpu(cdll):
    """ashrt_td_forward / ashrt_td_adjoint reject bad arguments before any CUDA
    call (the pointers are never dereferenced on these paths)."""
    v = (ctypes.c_float * 2)(1500.0, 2500.0)
    bad_v = (ctypes.c_float * 2)(1500.0, -1.0)
    t0 = (ctypes.c_float * 1)(-0.1,)
    buf = ctypes.c_void_p(16)                      # never dereferenced
    for fn in (cdll.ashrt_td_forward, cdll.ashrt_td_adjoint):
        assert fn(1, 8, 0.004, 12.5, v, 2, None, 1, buf, buf, 1, None) == 1
        assert fn(64, 8, 0.004, 12.5, bad_v, 2, None, 1, buf, buf, 1, None) == 1
        assert b"velocity 1" in cdll.ashrt_last_error()
        assert fn(64, 8, 0.004, 12.5, v, 2, t0, 1, buf, buf, 1, None) == 1
        assert b"shift 0" in cdll.ashrt_last_error()
        assert fn(64, 8, 0.004, 12.5, v, 2, None, 200, buf, buf, 1, None) == 1
        assert fn(64, 8, 0.004, 12.5, v, 2, None, 1, None, buf, 1, None) == 1
        assert fn(64, 8, -0.004, 12.5, v, 2, None, 1, buf, buf, 1, None) == 1


def test_solver_and_acquisition_argument_checks_without_gpu(cdll):
    """ashrt_fista and the blending / sorting calls reject bad arguments
    before any CUDA call."""
    from paper_1711_10214_gb300 import ashrt
    buf = ctypes.c_void_p(16)                      # never dereferenced
    assert cdll.ashrt_fista(None, buf, None, buf, buf, None, 1, None, None, None) == 1
    assert b"NULL plan" in cdll.ashrt_last_error()
    assert cdll.ashrt_blend(buf, 9000, 4, 64, buf, buf, 100, None) == 1      # too many shots
    assert cdll.ashrt_blend(buf, 8, 4, 64, None, buf, 100, None) == 1        # no firing times
    assert cdll.ashrt_pseudo_deblend(buf, 4, 0, buf, 8, 64, buf, None) == 1  # empty record
    assert cdll.ashrt_sort_gathers(buf, 3, 4, 8, buf, None) == 1             # in place
    assert b"distinct" in cdll.ashrt_last_error()
    o = ashrt.FistaOpts()
    cdll.fista_default_opts(ctypes.byref(o))
    assert (o.mu, o.n_iter, o.n_power) == (0.0, 50, 20)


def test_static_forward_and_quality_argument_checks_without_gpu(cdll):
    """ashrt_forward_static applies the plan's argument rules (t0_shifts NULL
    only with nt0 = 1, non-negative fmax and wavelet frequency) before any CUDA
    call; ashrt_quality_db and ashrt_fp32_peak reject bad sizes likewise."""
    from paper_1711_10214_gb300 import ashrt
    buf = ctypes.c_void_p(16)                      # never dereferenced
    v = (ctypes.c_float * 2)(1500.0, 2500.0)
    o = ashrt.AshrtOpts()
    cdll.ashrt_default_opts(ctypes.byref(o))
    fs = cdll.ashrt_forward_static
    assert fs(64, 16, 0.004, 12.5, v, 2, None, 3, ctypes.byref(o), buf, buf, None, 1, None) == 1
    assert b"nt0 = 1" in cdll.ashrt_last_error()
    for field in ("fmax_hz", "wavelet_peak_hz"):
        bad = ashrt.AshrtOpts()
        cdll.ashrt_default_opts(ctypes.byref(bad))
        for val in (-1.0, float("nan")):
            setattr(bad, field, val)
            assert fs(64, 16, 0.004, 12.5, v, 2, None, 1, ctypes.byref(bad), buf, buf, None, 1,
                      None) == 1
            assert b">= 0" in cdll.ashrt_last_error()
    sums = ctypes.c_void_p(32)
    assert cdll.ashrt_quality_db(buf, buf, 0, 10, sums, None, None) == 1
    assert cdll.ashrt_quality_db(buf, None, 2, 10, sums, None, None) == 1
    assert cdll.ashrt_quality_db(buf, buf, 2, 10, None, None, None) == 1
    t = ctypes.c_double()
    assert cdll.ashrt_fp32_peak(0, 1, ctypes.byref(t), None, None) == 1


def test_irregular_plan_argument_checks_without_gpu(cdll):
    """ashrt_plan_create_irregular rejects missing or non-finite trace
    positions and an empty trace set before any CUDA call."""
    h = ctypes.c_void_p()
    v = (ctypes.c_float * 1)(1500.0)
    x = (ctypes.c_double * 3)(0.0, 12.5, float("inf"))
    f = cdll.ashrt_plan_create_irregular
    assert f(ctypes.byref(h), 64, 8, 0.004, 12.5, v, 1, None, 1, None, 3, None) == 1
    assert b"trace_x" in cdll.ashrt_last_error()
    assert f(ctypes.byref(h), 64, 8, 0.004, 12.5, v, 1, None, 1, x, 0, None) == 1
    assert f(ctypes.byref(h), 64, 8, 0.004, 12.5, v, 1, None, 1, x, 3, None) == 1
    assert b"position 2" in cdll.ashrt_last_error() and h.value is None

"""The C ABI's error contract, checked without a GPU: arguments are checked before any CUDA call,
each failure returns its documented status, and rfd_last_error names the offending argument."""
import ctypes

import numpy as np
import pytest

ARG, SHAPE = -1, -2


@pytest.fixture(scope="module")
def lib():
    from paper_2601_18835_gb300 import build, _native
    build.build()
    return _native.load()


@pytest.fixture(scope="module")
def native():
    from paper_2601_18835_gb300 import _native
    return _native


def p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def plan_create(lib, native, options, ctx=None):
    g = native.Grid(2048.0, 4096, 20.0, 0, 0)
    ro, k = np.zeros(4, np.int32), np.full(4, 64, np.int32)
    h = ctypes.c_void_p()
    st = lib.rfd_plan_create_ex(ctx, ctypes.byref(g), 1, 4, p(ro), p(k), 1, 205, 25.0, 63,
                                ctypes.byref(options) if options is not None else None, ctypes.byref(h))
    return st, lib.rfd_last_error().decode(), h.value


@pytest.mark.parametrize("field,value,message", [
    ("long_k", 600, "long_k must be in [0, 512]"),
    ("long_k", -1, "long_k must be in [0, 512]"),
    ("fft_k", 5000, "fft_k must be in [0, 4096]"),
    ("out_len", 100, "out_len=100 must be 0 or a positive multiple of 512"),
    ("fft_rem", 64, "fft_rem must be in [0, 63]"),
    ("debug_flags", 2, "unknown debug_flags bits"),
    ("grid_ctas", -1, "grid_ctas must be >= 0"),
])
def test_plan_options_are_checked_first(lib, native, field, value, message):
    o = native.PlanOptions()
    lib.rfd_plan_options_default(ctypes.byref(o))
    setattr(o, field, value)
    st, err, h = plan_create(lib, native, o)
    assert st == ARG and err == message and h is None


@pytest.mark.parametrize("slot,value", [(0, 20), (0, 144), (1, 80), (2, 48), (2, 0)])
def test_tile_sizes_are_checked(lib, native, slot, value):
    o = native.PlanOptions()
    lib.rfd_plan_options_default(ctypes.byref(o))
    o.tile_nt[slot] = value
    st, err, _ = plan_create(lib, native, o)
    assert st == ARG and err.startswith("tile_nt[%d]=%d must be a multiple of 16" % (slot, value))


def test_valid_options_then_a_missing_context(lib, native):
    o = native.PlanOptions()
    lib.rfd_plan_options_default(ctypes.byref(o))
    assert plan_create(lib, native, o)[:2] == (ARG, "NULL ctx or out")
    assert plan_create(lib, native, None)[:2] == (ARG, "NULL ctx or out")


def test_entry_points_refuse_a_missing_context(lib, native):
    g = native.Grid(2048.0, 4096, 20.0, 0, 0)
    n, cnt, h = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_void_p()
    calls = {
        "rfd_find_triggers": lambda: lib.rfd_find_triggers(None, 4, None, ctypes.byref(cnt), 0, None, 0,
                                                           ctypes.byref(n), None),
        "rfd_make_taps": lambda: lib.rfd_make_taps(None, ctypes.byref(g), None, None, 1, None, None, 0, None, None,
                                                   0, 0.999, 64, 0.1, None, None, None, None, None, None),
        "rfd_filter_reference": lambda: lib.rfd_filter_reference(None, ctypes.byref(g), None, None, None, 1, 63, 1,
                                                                 None, None, None),
        "rfd_gen_templates": lambda: lib.rfd_gen_templates(None, ctypes.byref(g), None, 1, None, None),
        "rfd_ifft_c2c": lambda: lib.rfd_ifft_c2c(None, 4096, 1, None, None, None),
    }
    for name, call in calls.items():
        assert call() == ARG, name
        assert lib.rfd_last_error() == b"ctx is NULL", name
    for name, call in {
        "rfd_mlp_create": lambda: lib.rfd_mlp_create(None, ctypes.byref(g), None, None, 1, ctypes.byref(h)),
        "rfd_subband_create": lambda: lib.rfd_subband_create(None, ctypes.byref(g), None, None, 1, 8,
                                                             ctypes.byref(h)),
        "rfd_make_taps_cached": lambda: lib.rfd_make_taps_cached(None, None, ctypes.byref(g), None, None, 1, None,
                                                                 None, 1, None, None, 0, 0.999, 64, 0.1, None, None,
                                                                 None, None, None, None, None),
    }.items():
        assert call() == ARG and lib.rfd_last_error() == b"NULL argument", name


@pytest.mark.parametrize("n_tmpl,cap,tcap,status,message", [
    (0, 0, 0, SHAPE, "n_tmpl=0 outside [1, 32768]"),
    (32769, 0, 0, SHAPE, "n_tmpl=32769 outside [1, 32768]"),
    (4, 131073, 0, SHAPE, "cand_capacity=131073 outside [0, 131072]"),
    (4, 0, -1, SHAPE, "negative trigger capacity"),
])
def test_no_allocation_merge_limits(lib, n_tmpl, cap, tcap, status, message):
    n, cnt = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.rfd_find_triggers_noalloc(n_tmpl, None, ctypes.byref(cnt), cap, None, tcap, ctypes.byref(n), None)
    assert st == status and message in lib.rfd_last_error().decode()


def test_no_allocation_merge_needs_its_count(lib):
    n = ctypes.c_int64(0)
    assert lib.rfd_find_triggers_noalloc(4, None, None, 0, None, 0, ctypes.byref(n), None) == ARG
    assert lib.rfd_last_error() == b"NULL argument"


def test_every_status_has_its_own_message(lib):
    msgs = [lib.rfd_status_string(s) for s in range(-7, 1)]
    assert len(set(msgs)) == len(msgs) and all(msgs)
    assert lib.rfd_status_string(0) == b"ok" and lib.rfd_status_string(-8) == b"unknown status"

"""CPU checks of the C ABI: librfd.so builds, loads, exports every function declared in
include/rfd.h, and its host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_18835_gb300 import build, _native
    build.build()
    return _native.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rfd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rfd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rfd_make_taps", "rfd_filter_reference", "rfd_ratio_filter_batch", "rfd_find_triggers"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_declares_every_exported_function(lib):
    from paper_2601_18835_gb300 import _native
    assert set(declared_functions()) == set(_native.SIGNATURES)


def test_host_only_entry_points(lib):
    import re
    header = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                               "rfd.h")).read()
    assert lib.rfd_version() == int(re.search(r"#define RFD_VERSION (\d+)", header).group(1))
    assert lib.rfd_status_string(-7) == b"output capacity exceeded"
    assert lib.rfd_qref_ld(524288, 127) == 524288 + 128
    assert lib.rfd_qref_ld(16384, 0) == 16384
    assert lib.rfd_qref_ld(1024, 1) == 1088


def test_ctx_create_without_gpu_reports_an_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.rfd_ctx_create(0, ctypes.byref(h))
    assert st != 0
    assert h.value is None
    assert len(lib.rfd_last_error()) > 0


def test_struct_layouts():
    from paper_2601_18835_gb300 import _native
    assert ctypes.sizeof(_native.Grid) == 32
    assert ctypes.sizeof(_native.Params) == 40
    assert _native.CANDIDATE_DTYPE.itemsize == 24
    assert _native.TRIGGER_DTYPE.itemsize == 20

"""ctypes declarations of the librfd C ABI (include/rfd.h).

Loading fails loudly when librfd.so has not been built: there is no fallback path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librfd.so")

RFD_OK = 0
RFD_ERR_ARG = -1
RFD_ERR_SHAPE = -2
RFD_ERR_UNSUPPORTED = -3
RFD_ERR_CUDA = -4
RFD_ERR_NOMEM = -5
RFD_ERR_TIMEOUT = -6
RFD_ERR_OVERFLOW = -7

PN_SO = 1
PN_TIDAL = 2
PREC_FP32 = 0
PREC_FP16X3 = 1
PREC_BF16X3 = 2
NOALLOC_MAX_TEMPLATES = 32768
NOALLOC_MAX_CANDIDATES = 131072


class Grid(ctypes.Structure):
    _fields_ = [("fs", ctypes.c_double), ("n", ctypes.c_int64), ("f_low", ctypes.c_double),
                ("pn_flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class PlanOptions(ctypes.Structure):
    _fields_ = [("tile_nt", ctypes.c_int32 * 3), ("mix_k", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("long_k", ctypes.c_int32), ("fft_k", ctypes.c_int32), ("out_len", ctypes.c_int32),
                ("fft_rem", ctypes.c_int32), ("debug_flags", ctypes.c_int32)]


DEBUG_STALL_TAPS = 1


class Params(ctypes.Structure):
    _fields_ = [("m1", ctypes.c_double), ("m2", ctypes.c_double), ("chi1", ctypes.c_double),
                ("chi2", ctypes.c_double), ("lambda_tilde", ctypes.c_double)]


CANDIDATE_DTYPE = np.dtype([("key", "<u8"), ("j", "<u4"), ("w", "<u4"), ("zr", "<f4"), ("zi", "<f4")])
TRIGGER_DTYPE = np.dtype([("j", "<i4"), ("t", "<i4"), ("snr2", "<f4"), ("zr", "<f4"), ("zi", "<f4")])
assert CANDIDATE_DTYPE.itemsize == 24 and TRIGGER_DTYPE.itemsize == 20

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_flt = ctypes.c_float

# name -> (restype, argtypes)
SIGNATURES = {
    "rfd_version": (_i32, []),
    "rfd_status_string": (ctypes.c_char_p, [_i32]),
    "rfd_last_error": (ctypes.c_char_p, []),
    "rfd_kernel_launches": (_i64, []),
    "rfd_ctx_create": (_i32, [_i32, ctypes.POINTER(_vp)]),
    "rfd_ctx_destroy": (None, [_vp]),
    "rfd_ctx_trim": (None, [_vp]),
    "rfd_qref_ld": (_i64, [_i64, _i32]),
    "rfd_gen_templates": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _i32, _vp, _vp]),
    "rfd_make_taps": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp, _i32, _dbl,
                             _i32, _dbl, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rfd_filter_reference": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp,
                                    _vp]),  # href_dev is a device pointer
    "rfd_plan_create": (_i32, [_vp, ctypes.POINTER(Grid), _i32, _i32, _vp, _vp, _i32, _i32, _flt, _i32,
                               ctypes.POINTER(_vp)]),
    "rfd_plan_destroy": (None, [_vp]),
    "rfd_plan_set_taps": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp]),
    "rfd_plan_executed_flops": (_dbl, [_vp]),
    "rfd_plan_template_kernels": (_i32, [_vp, _vp]),
    "rfd_plan_options_default": (None, [_vp]),
    "rfd_plan_create_ex": (_i32, [_vp, ctypes.POINTER(Grid), _i32, _i32, _vp, _vp, _i32, _i32, _flt, _i32, _vp,
                                  ctypes.POINTER(_vp)]),
    "rfd_search_create": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _i64, _vp,
                                 ctypes.POINTER(_vp)]),
    "rfd_search_run": (_i32, [_vp, _vp, ctypes.POINTER(_i64)]),
    "rfd_search_run_at": (_i32, [_vp, _i64, _vp, ctypes.POINTER(_i64)]),
    "rfd_search_run_host": (_i32, [_vp, _vp, _vp, _i64, _vp, ctypes.POINTER(_i64)]),
    "rfd_search_kernels_per_run": (_i64, [_vp]),
    "rfd_search_filter_ms": (_dbl, [_vp]),
    "rfd_search_step_ms": (_dbl, [_vp]),
    "rfd_search_destroy": (None, [_vp]),
    "rfd_ratio_filter_batch": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "rfd_ratio_filter_window": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "rfd_find_triggers": (_i32, [_vp, _i32, _vp, _vp, _i64, _vp, _i64, ctypes.POINTER(_i64), _vp]),
    "rfd_find_triggers_noalloc": (_i32, [_i32, _vp, _vp, _i64, _vp, _i64, ctypes.POINTER(_i64), _vp]),
    "rfd_findchirp": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _vp, _vp, _i32, _i32, _flt, _vp, _i64, _vp,
                             _vp]),
    "rfd_ifft_c2c": (_i32, [_vp, _i64, _i32, _vp, _vp, _vp]),
    "rfd_fft_c2c": (_i32, [_vp, _i64, _i32, _i32, _i32, _vp, _vp, _vp]),
    "rfd_make_taps_at_lag": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp, _i32,
                                    _dbl, _vp, _vp, _vp, _vp]),
    "rfd_taps_key": (_i32, [ctypes.POINTER(Grid), _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp, _i32, _dbl, _i32, _dbl,
                            _vp]),
    "rfd_make_taps_cached": (_i32, [ctypes.c_char_p, _vp, ctypes.POINTER(Grid), _vp, _vp, _i32, _vp, _vp, _i32, _vp,
                                    _vp, _i32, _dbl, _i32, _dbl, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_i32), _vp]),
    "rfd_make_taps_fit": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp, _i32, _dbl,
                                 _dbl, _i32, _dbl, _vp, _vp, _vp, _vp, _vp, _vp]),
    "rfd_subband_create": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _vp, _i32, _i32, ctypes.POINTER(_vp)]),
    "rfd_subband_destroy": (None, [_vp]),
    "rfd_subband_edges": (_i32, [_vp, _vp]),
    "rfd_subband_filter_reference": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "rfd_subband_shares": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _vp, _i32, _vp, _vp]),
    "rfd_subband_chi2": (_i32, [_vp, _vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _i64, _vp, _vp, _vp]),
    "rfd_mlp_param_count": (_i64, []),
    "rfd_mlp_create": (_i32, [_vp, ctypes.POINTER(Grid), _vp, _vp, _i32, ctypes.POINTER(_vp)]),
    "rfd_mlp_destroy": (None, [_vp]),
    "rfd_mlp_set_weights": (_i32, [_vp, _vp]),
    "rfd_mlp_get_weights": (_i32, [_vp, _vp]),
    "rfd_mlp_set_norm": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "rfd_mlp_get_autocorr": (_i32, [_vp, _vp]),
    "rfd_mlp_features": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "rfd_mlp_train_step": (_i32, [_vp, _vp, _vp, _i32, _vp, _i32, _flt, _vp]),
    "rfd_mlp_grads": (_i32, [_vp, _vp, _vp, _i32, _vp, _i32, _vp, _vp, _vp]),
    "rfd_mlp_state": (_i32, [_vp, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_flt), _vp]),
    "rfd_mlp_save": (_i32, [_vp, ctypes.c_char_p, _vp]),
    "rfd_mlp_load": (_i32, [_vp, ctypes.c_char_p, _vp]),
    "rfd_mlp_infer": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp]),
    "rfd_mlp_cross_match": (_i32, [_vp, _vp, _i32, _vp, _i64, _vp, _i64, _vp, _vp]),
    "rfd_learned_taps": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _dbl, _i32, _dbl, _vp, _vp, _vp, _vp, _vp, _vp,
                                _vp]),
}
MLP_TAPS = 128
MLP_FEATURES_LD = 64

_lib = None


def load(path: str = LIB_PATH):
    """Load librfd.so and declare every entry point.  Raises if the library is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("librfd.so is not built (%s); build it with __graft_entry__.build() "
                          "or python paper_2601_18835_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RfdError(RuntimeError):
    def __init__(self, status, msg, needed=None):
        super().__init__("librfd status %d: %s" % (status, msg))
        self.status = status
        self.needed = needed


def check(status, needed=None):
    if status != RFD_OK:
        lib = load()
        raise RfdError(status, lib.rfd_last_error().decode(errors="replace"), needed)

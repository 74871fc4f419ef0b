"""Ratio-Filter Dechirping on GB300: Python binding over the librfd C ABI.

The binding only marshals arguments (torch tensors for device memory, torch streams); every
step of the method runs in the library's CUDA kernels.  Names follow include/rfd.h:

  gen_templates      TaylorF2 templates h(f) (FP64 phase)                      Eq. 1
  make_taps          ratio-filter taps, lags, sigma_eff, match                 Eqs. 2-3, Sec. V, Eqs. 5-6
  filter_reference   reference SNR series q_ref (pointwise + Stockham IFFT)    Eqs. 1, 3
  Plan.ratio_filter_batch   FIR of every template on q_ref + fused triggers    Eq. 3, Table II
  find_triggers      per-window maxima above threshold                         Table II
  findchirp          the FINDCHIRP comparison path                             Eq. 1
  make_taps_at_lag   taps at a given lag (the learned-tap targets)             Sec. V
  Mlp                learned taps: per-reference networks, training, inference Eq. 4 through Eqs. 5-6
"""
import ctypes
import os

import numpy as np
import torch

from . import _native
from ._native import (CANDIDATE_DTYPE, PN_SO, PN_TIDAL, PREC_BF16X3, PREC_FP16X3, PREC_FP32,  # noqa: F401
                      TRIGGER_DTYPE, RfdError, check)

__all__ = ["Context", "Plan", "Search", "Mlp", "Subband", "grid", "gen_templates", "make_taps", "make_taps_fit",
           "make_taps_at_lag",
           "make_taps_cached", "taps_key", "filter_reference",
           "find_triggers", "find_triggers_noalloc", "findchirp", "ifft_c2c", "qref_ld", "candidates_to_numpy",
           "triggers_to_numpy", "CANDIDATE_DTYPE", "TRIGGER_DTYPE"]


def _lib():
    return _native.load()


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return ctypes.c_void_p(t.data_ptr())
    return t


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def grid(fs, n, f_low, pn_flags=0):
    return _native.Grid(float(fs), int(n), float(f_low), int(pn_flags), 0)


def _params(p):
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64).reshape(-1, 5))
    arr = (_native.Params * max(1, len(p)))()
    ctypes.memmove(arr, p.ctypes.data, p.nbytes)
    return arr, len(p)


def _i32_host(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def kernel_launches():
    """Kernels launched by librfd in this process so far."""
    return int(_lib().rfd_kernel_launches())


def qref_ld(n, halo):
    return int(_lib().rfd_qref_ld(int(n), int(halo)))


class Context:
    """A librfd context on one CUDA device (FFT tables and workspaces)."""

    def __init__(self, device=0):
        lib = _lib()
        h = ctypes.c_void_p()
        check(lib.rfd_ctx_create(int(device), ctypes.byref(h)))
        self.handle = h
        self.device = int(device)

    def trim(self):
        """Free the scratch workspaces (re-created on demand)."""
        _lib().rfd_ctx_trim(self.handle)

    def close(self):
        if self.handle:
            _lib().rfd_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gen_templates(ctx, g, params, out, stream=None):
    pa, n = _params(params)
    check(_lib().rfd_gen_templates(ctx.handle, ctypes.byref(g), pa, n, _ptr(out), _stream(stream)))
    return out


def make_taps(ctx, g, psd, refs, tmpl, ref_of, k, k_stride, alpha, taps, lag, sigma, match=None,
              stream=None, buckets=None, energy_frac=0.999, k_out=None):
    """k: taps per template (array), or None to choose each K from `buckets` (the smallest
    bucket whose best window holds `energy_frac` of the impulse response's energy); the
    chosen K is written to k_out (device int32)."""
    ra, nr = _params(refs)
    ta, nt = _params(tmpl)
    ro, rop = _i32_host(ref_of)
    if k is None:
        kp = None
        bk, bkp = _i32_host(buckets)
        nbk = len(bk)
    else:
        kk, kp = _i32_host(k)
        bkp, nbk = None, 0
    check(_lib().rfd_make_taps(ctx.handle, ctypes.byref(g), _ptr(psd), ra, nr, ta, rop, nt, kp, bkp, nbk,
                               float(energy_frac), int(k_stride), float(alpha), _ptr(taps), _ptr(k_out),
                               _ptr(lag), _ptr(sigma), _ptr(match), _stream(stream)))


def _k_policy(k, buckets):
    """(array kept alive by the caller, k pointer, bucket pointer, bucket count)."""
    if k is None:
        bk, bkp = _i32_host(buckets)
        return bk, None, bkp, len(bk)
    kk, kp = _i32_host(k)
    return kk, kp, None, 0


def taps_key(g, psd, refs, tmpl, ref_of, k, k_stride, alpha, buckets=None, energy_frac=0.999):
    """SHA-256 digest (32 bytes) of a tap bank's inputs (rfd_taps_key); psd: host float64 [n/2+1]."""
    ra, nr = _params(refs)
    ta, nt = _params(tmpl)
    ro, rop = _i32_host(ref_of)
    keep, kp, bkp, nbk = _k_policy(k, buckets)
    ps = np.ascontiguousarray(np.asarray(psd, dtype=np.float64))
    out = (ctypes.c_uint8 * 32)()
    check(_lib().rfd_taps_key(ctypes.byref(g), ps.ctypes.data_as(ctypes.c_void_p), ra, nr, ta, rop, nt, kp, bkp, nbk,
                              float(energy_frac), int(k_stride), float(alpha), out))
    return bytes(out)


def make_taps_cached(cache_dir, ctx, g, psd, refs, tmpl, ref_of, k, k_stride, alpha, taps, lag, sigma, match=None,
                     stream=None, buckets=None, energy_frac=0.999, k_out=None):
    """make_taps through the tap-bank files under cache_dir (rfd_make_taps_cached).  Returns True
    when the taps were read from a file, False when they were extracted (and stored)."""
    ra, nr = _params(refs)
    ta, nt = _params(tmpl)
    ro, rop = _i32_host(ref_of)
    keep, kp, bkp, nbk = _k_policy(k, buckets)
    hit = ctypes.c_int32(0)
    check(_lib().rfd_make_taps_cached(os.fsencode(cache_dir), ctx.handle, ctypes.byref(g), _ptr(psd), ra, nr, ta,
                                      rop, nt, kp, bkp, nbk, float(energy_frac), int(k_stride), float(alpha),
                                      _ptr(taps), _ptr(k_out), _ptr(lag), _ptr(sigma), _ptr(match),
                                      ctypes.byref(hit), _stream(stream)))
    return bool(hit.value)


def make_taps_fit(ctx, g, psd, refs, tmpl, ref_of, k, k_stride, alpha, taps, lag, sigma, match, ridge=1e-6,
                  buckets=None, match_target=0.99, k_out=None, stream=None):
    """Chi^2-fitted taps (Sec. V.A): k per template, or k=None with buckets and a target match."""
    ra, nr = _params(refs)
    ta, nt = _params(tmpl)
    ro, rop = _i32_host(ref_of)
    if k is None:
        kp = None
        bk, bkp = _i32_host(buckets)
        nbk = len(bk)
    else:
        kk, kp = _i32_host(k)
        bkp, nbk = None, 0
    check(_lib().rfd_make_taps_fit(ctx.handle, ctypes.byref(g), _ptr(psd), ra, nr, ta, rop, nt, kp, bkp, nbk,
                                   float(match_target), float(ridge), int(k_stride), float(alpha), _ptr(taps),
                                   _ptr(k_out), _ptr(lag), _ptr(sigma), _ptr(match), _stream(stream)))


def make_taps_at_lag(ctx, g, psd, refs, tmpl, ref_of, k, lag, k_stride, alpha, taps, sigma, match=None,
                     stream=None):
    """Taps placed at the given lags (int32 per template, in [-n/2, n/2))."""
    ra, nr = _params(refs)
    ta, nt = _params(tmpl)
    ro, rop = _i32_host(ref_of)
    kk, kp = _i32_host(k)
    ll, lp = _i32_host(lag)
    check(_lib().rfd_make_taps_at_lag(ctx.handle, ctypes.byref(g), _ptr(psd), ra, nr, ta, rop, nt, kp, lp,
                                      int(k_stride), float(alpha), _ptr(taps), _ptr(sigma), _ptr(match),
                                      _stream(stream)))


def filter_reference(ctx, g, dtilde, psd, href, halo, precision, qref, qscale, stream=None):
    """href: complex64 [n_ref, n/2+1] reference templates (from gen_templates)."""
    check(_lib().rfd_filter_reference(ctx.handle, ctypes.byref(g), _ptr(dtilde), _ptr(psd), _ptr(href),
                                      int(href.shape[0]), int(halo), int(precision), _ptr(qref), _ptr(qscale),
                                      _stream(stream)))


class Plan:
    """One bank's ratio-filter schedule (templates tiled per reference) and packed taps."""

    def __init__(self, ctx, g, n_ref, ref_of, k, precision, window, threshold, halo, options=None):
        """options: dict with any of tile_nt (3 ints), mix_k (0/1), grid_ctas (int), long_k (int),
        fft_k (int: templates with fft_k < K <= 1024 use the block-FFT kernel), out_len (int: outputs per
        call, a multiple of 512; 0 = the whole segment), fft_rem (int: a reference's last long-kernel
        tile of at most this many templates goes to the block-FFT kernel), debug_flags (testing only)."""
        ro, rop = _i32_host(ref_of)
        kk, kp = _i32_host(k)
        h = ctypes.c_void_p()
        opt = None
        if options:
            opt = _native.PlanOptions()
            _lib().rfd_plan_options_default(ctypes.byref(opt))
            if "tile_nt" in options:
                for i, v in enumerate(options["tile_nt"]):
                    opt.tile_nt[i] = int(v)
            if "mix_k" in options:
                opt.mix_k = int(options["mix_k"])
            if "grid_ctas" in options:
                opt.grid_ctas = int(options["grid_ctas"])
            if "long_k" in options:
                opt.long_k = int(options["long_k"])
            if "fft_k" in options:
                opt.fft_k = int(options["fft_k"])
            if "out_len" in options:
                opt.out_len = int(options["out_len"])
            if "fft_rem" in options:
                opt.fft_rem = int(options["fft_rem"])
            if "debug_flags" in options:
                opt.debug_flags = int(options["debug_flags"])
        check(_lib().rfd_plan_create_ex(ctx.handle, ctypes.byref(g), int(n_ref), len(ro), rop, kp,
                                        int(precision), int(window), float(threshold), int(halo),
                                        ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
        self.options = dict(options or {})
        self.handle = h
        self.ctx = ctx
        self.n_tmpl = len(ro)

    def template_kernels(self):
        """Per template, the kernel that filters it: 0 FP32 direct FIR, 1 tensor cores with time
        on M, 2 tensor cores with templates on M, 3 block FFT (rfd_plan_template_kernels)."""
        out = np.empty(self.n_tmpl, dtype=np.int32)
        check(_lib().rfd_plan_template_kernels(self.handle, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_taps(self, taps, k_stride, lag, sigma, stream=None):
        check(_lib().rfd_plan_set_taps(self.handle, _ptr(taps), int(k_stride), _ptr(lag), _ptr(sigma),
                                       _stream(stream)))

    def ratio_filter_batch(self, qref, qscale, cand, cand_count, stream=None):
        cap = cand.numel() * cand.element_size() // CANDIDATE_DTYPE.itemsize
        check(_lib().rfd_ratio_filter_batch(self.handle, _ptr(qref), _ptr(qscale), _ptr(cand), int(cap),
                                            _ptr(cand_count), _stream(stream)))

    def ratio_filter_window(self, qref, qscale, u_begin, cand, cand_count, stream=None):
        """The plan's out_len outputs from the position held in u_begin (int64 device tensor)."""
        cap = cand.numel() * cand.element_size() // CANDIDATE_DTYPE.itemsize
        check(_lib().rfd_ratio_filter_window(self.handle, _ptr(qref), _ptr(qscale), _ptr(u_begin), _ptr(cand),
                                             int(cap), _ptr(cand_count), _stream(stream)))

    def executed_flops(self):
        """Flops one ratio_filter_batch call executes (tensor-core or FMA)."""
        return float(_lib().rfd_plan_executed_flops(self.handle))

    def close(self):
        if self.handle:
            _lib().rfd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Search:
    """One segment through filter_reference, ratio_filter_batch and the trigger merge, captured
    once into a CUDA graph (rfd_search_*); buffers are bound at creation.  `stream` must be a
    torch.cuda.Stream other than the default stream."""

    def __init__(self, plan, dtilde, psd, href, qref, qscale, cand, cand_count, trig, stream):
        cap = cand.numel() * cand.element_size() // CANDIDATE_DTYPE.itemsize
        tcap = trig.numel() * trig.element_size() // TRIGGER_DTYPE.itemsize
        h = ctypes.c_void_p()
        self.stream = stream
        check(_lib().rfd_search_create(plan.handle, _ptr(dtilde), _ptr(psd), _ptr(href), _ptr(qref), _ptr(qscale),
                                       _ptr(cand), int(cap), _ptr(cand_count), _ptr(trig), int(tcap),
                                       _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.plan = plan

    @property
    def kernels_per_run(self):
        return int(_lib().rfd_search_kernels_per_run(self.handle))

    def step_ms(self):
        """Device time of the whole last run (events at the graph's first and last node)."""
        return float(_lib().rfd_search_step_ms(self.handle))

    def filter_ms(self):
        """Device time of the ratio-filter kernel in the last run (events inside the graph)."""
        return float(_lib().rfd_search_filter_ms(self.handle))

    def run(self, u_begin=None):
        """Replays the graph, waits, returns the number of triggers.  u_begin: the window start
        for a plan with out_len < n (streaming)."""
        n = ctypes.c_int64(0)
        if u_begin is None:
            check(_lib().rfd_search_run(self.handle, _stream(self.stream), ctypes.byref(n)), needed=n.value)
        else:
            check(_lib().rfd_search_run_at(self.handle, int(u_begin), _stream(self.stream), ctypes.byref(n)),
                  needed=n.value)
        return int(n.value)

    def run_host(self, dtilde_host, trig_host):
        """One segment end to end from host memory (rfd_search_run_host): dtilde_host (a CPU
        complex64 tensor of n/2+1 bins, pinned for an asynchronous copy) in, triggers out into
        trig_host (a CPU uint8 tensor of rfd_trigger records).  Returns the number of triggers."""
        for t in (dtilde_host, trig_host):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError("expected contiguous host (CPU) tensors")
        tcap = trig_host.numel() * trig_host.element_size() // TRIGGER_DTYPE.itemsize
        n = ctypes.c_int64(0)
        check(_lib().rfd_search_run_host(self.handle, ctypes.c_void_p(dtilde_host.data_ptr()),
                                         ctypes.c_void_p(trig_host.data_ptr()), int(tcap), _stream(self.stream),
                                         ctypes.byref(n)), needed=n.value)
        return int(n.value)

    def close(self):
        if self.handle:
            _lib().rfd_search_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def find_triggers(ctx, n_tmpl, cand, cand_count, trig, stream=None):
    """Returns the number of triggers written to `trig` (synchronises the stream)."""
    cap = cand.numel() * cand.element_size() // CANDIDATE_DTYPE.itemsize
    tcap = trig.numel() * trig.element_size() // TRIGGER_DTYPE.itemsize
    n = ctypes.c_int64(0)
    st = _lib().rfd_find_triggers(ctx.handle, int(n_tmpl), _ptr(cand), _ptr(cand_count), int(cap),
                                  _ptr(trig), int(tcap), ctypes.byref(n), _stream(stream))
    check(st, needed=n.value)
    return int(n.value)


def find_triggers_noalloc(n_tmpl, cand, cand_count, trig, stream=None):
    """find_triggers without any device allocation (static scratch, fixed maximum sizes);
    runs on the current CUDA device.  Returns the number of triggers."""
    cap = cand.numel() * cand.element_size() // CANDIDATE_DTYPE.itemsize
    tcap = trig.numel() * trig.element_size() // TRIGGER_DTYPE.itemsize
    n = ctypes.c_int64(0)
    st = _lib().rfd_find_triggers_noalloc(int(n_tmpl), _ptr(cand), _ptr(cand_count), int(cap), _ptr(trig),
                                          int(tcap), ctypes.byref(n), _stream(stream))
    check(st, needed=n.value)
    return int(n.value)


def findchirp(ctx, g, dtilde, psd, h, window, threshold, cand, cand_count, stream=None):
    """h: complex64 [n_tmpl, n/2+1] templates (from gen_templates)."""
    cap = cand.numel() * cand.element_size() // CANDIDATE_DTYPE.itemsize
    check(_lib().rfd_findchirp(ctx.handle, ctypes.byref(g), _ptr(dtilde), _ptr(psd), _ptr(h), int(h.shape[0]),
                               int(window), float(threshold), _ptr(cand), int(cap), _ptr(cand_count),
                               _stream(stream)))


def ifft_c2c(ctx, x, out, stream=None):
    n = x.shape[-1]
    batch = x.numel() // n
    check(_lib().rfd_ifft_c2c(ctx.handle, int(n), int(batch), _ptr(x), _ptr(out), _stream(stream)))
    return out


def fft_c2c(ctx, x, out, inverse, stream=None):
    """Unnormalised FFT of the rows of x (complex64 or complex128, last axis a power of two)."""
    n = x.shape[-1]
    batch = x.numel() // n
    assert x.dtype == out.dtype and x.dtype in (torch.complex64, torch.complex128)
    check(_lib().rfd_fft_c2c(ctx.handle, int(n), int(batch), int(x.dtype == torch.complex128), int(bool(inverse)),
                             _ptr(x), _ptr(out), _stream(stream)))
    return out


def candidates_to_numpy(buf, count):
    raw = buf[: count * CANDIDATE_DTYPE.itemsize].cpu().numpy().view(np.uint8)
    return raw.view(CANDIDATE_DTYPE)


def triggers_to_numpy(buf, count):
    raw = buf[: count * TRIGGER_DTYPE.itemsize].cpu().numpy().view(np.uint8)
    return raw.view(TRIGGER_DTYPE)


class Mlp:
    """Learned taps: one network per reference (include/rfd.h, "learned taps")."""

    TAPS = _native.MLP_TAPS
    FEATURES_LD = _native.MLP_FEATURES_LD

    def __init__(self, ctx, g, psd, refs):
        ra, nr = _params(refs)
        h = ctypes.c_void_p()
        check(_lib().rfd_mlp_create(ctx.handle, ctypes.byref(g), _ptr(psd), ra, nr, ctypes.byref(h)))
        self.handle = h
        self.n_ref = nr
        self.ctx = ctx

    @staticmethod
    def param_count():
        return int(_lib().rfd_mlp_param_count())

    def set_weights(self, w):
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32).reshape(self.n_ref, self.param_count()))
        check(_lib().rfd_mlp_set_weights(self.handle, w.ctypes.data_as(ctypes.c_void_p)))

    def get_weights(self):
        w = np.empty((self.n_ref, self.param_count()), dtype=np.float32)
        check(_lib().rfd_mlp_get_weights(self.handle, w.ctypes.data_as(ctypes.c_void_p)))
        return w

    def set_norm(self, mu, sd, out_scale, lag):
        mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float64).reshape(self.n_ref, 4))
        sd = np.ascontiguousarray(np.asarray(sd, dtype=np.float64).reshape(self.n_ref, 4))
        sc = np.ascontiguousarray(np.asarray(out_scale, dtype=np.float64).reshape(self.n_ref))
        lg, lp = _i32_host(np.asarray(lag).reshape(self.n_ref))
        check(_lib().rfd_mlp_set_norm(self.handle, mu.ctypes.data_as(ctypes.c_void_p),
                                      sd.ctypes.data_as(ctypes.c_void_p), sc.ctypes.data_as(ctypes.c_void_p), lp))

    def autocorr(self):
        c = np.empty((self.n_ref, 2 * self.TAPS - 1, 2), dtype=np.float64)
        check(_lib().rfd_mlp_get_autocorr(self.handle, c.ctypes.data_as(ctypes.c_void_p)))
        return c[..., 0] + 1j * c[..., 1]

    def features(self, params, net_of, out=None, stream=None):
        pa, n = _params(params)
        no, nop = _i32_host(net_of)
        if out is None:
            out = torch.empty((n, self.FEATURES_LD), dtype=torch.float16, device="cuda")
        check(_lib().rfd_mlp_features(self.handle, pa, nop, n, _ptr(out), _stream(stream)))
        return out

    def train_step(self, feat, target, n_train, idx, batch, lr, stream=None):
        check(_lib().rfd_mlp_train_step(self.handle, _ptr(feat), _ptr(target), int(n_train), _ptr(idx), int(batch),
                                        float(lr), _stream(stream)))

    def grads(self, feat, target, n_train, idx, batch, stream=None):
        g = torch.empty((self.n_ref, self.param_count()), dtype=torch.float32, device="cuda")
        loss = torch.empty(self.n_ref, dtype=torch.float32, device="cuda")
        check(_lib().rfd_mlp_grads(self.handle, _ptr(feat), _ptr(target), int(n_train), _ptr(idx), int(batch),
                                   _ptr(g), _ptr(loss), _stream(stream)))
        return g, loss

    def state(self, stream=None):
        """(per-network batch loss, steps taken, loss scale) after the last step."""
        loss = np.empty(self.n_ref, dtype=np.float32)
        step = ctypes.c_int32()
        scale = ctypes.c_float()
        check(_lib().rfd_mlp_state(self.handle, loss.ctypes.data_as(ctypes.c_void_p), ctypes.byref(step),
                                   ctypes.byref(scale), _stream(stream)))
        return loss, int(step.value), float(scale.value)

    def save(self, path, stream=None):
        """Checkpoint of the training state (weights, Adam moments, normalisation, lags,
        optimiser state) to `path` (rfd_mlp_save)."""
        check(_lib().rfd_mlp_save(self.handle, str(path).encode(), _stream(stream)))

    def load(self, path, stream=None):
        """Restores a checkpoint written for the same grid, PSD and references (rfd_mlp_load)."""
        check(_lib().rfd_mlp_load(self.handle, str(path).encode(), _stream(stream)))

    def infer(self, params, net_of, taps, lag, sigma, k_stride=None, stream=None):
        pa, n = _params(params)
        no, nop = _i32_host(net_of)
        ks = int(taps.shape[-1]) if k_stride is None else int(k_stride)
        check(_lib().rfd_mlp_infer(self.handle, pa, nop, n, ks, _ptr(taps), _ptr(lag), _ptr(sigma),
                                   _stream(stream)))

    def cross_match(self, net_of, rho1, rho2, stream=None):
        no, nop = _i32_host(net_of)
        out = torch.empty(len(no), dtype=torch.float64, device="cuda")
        check(_lib().rfd_mlp_cross_match(self.handle, nop, len(no), _ptr(rho1), int(rho1.shape[-1]), _ptr(rho2),
                                         int(rho2.shape[-1]), _ptr(out), _stream(stream)))
        return out

    def learned_taps(self, psd, tmpl, ref_of, taps, lag, sigma, spot_stride=8, min_match=0.999, alpha=0.1,
                     stream=None):
        """Surrogate taps with spot checks and exact fallback; returns (source, surrogate match, stats)."""
        ta, nt = _params(tmpl)
        ro, rop = _i32_host(ref_of)
        source = torch.empty(nt, dtype=torch.int32, device="cuda")
        smatch = torch.empty(nt, dtype=torch.float64, device="cuda")
        stats = np.zeros(4, dtype=np.int64)
        check(_lib().rfd_learned_taps(self.handle, _ptr(psd), ta, rop, nt, int(spot_stride), float(min_match),
                                      int(taps.shape[-1]), float(alpha), _ptr(taps), _ptr(lag), _ptr(sigma),
                                      _ptr(smatch), _ptr(source), stats.ctypes.data_as(ctypes.c_void_p),
                                      _stream(stream)))
        return source, smatch, {"surrogate": int(stats[0]), "exact": int(stats[1]), "spot_checked": int(stats[2]),
                                "spot_failed": int(stats[3])}

    def close(self):
        if self.handle:
            _lib().rfd_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Subband:
    """Sub-band chi^2 through the ratio filter (include/rfd.h, "sub-band chi^2")."""

    def __init__(self, ctx, g, psd, refs, p=8):
        ra, nr = _params(refs)
        h = ctypes.c_void_p()
        check(_lib().rfd_subband_create(ctx.handle, ctypes.byref(g), _ptr(psd), ra, nr, int(p), ctypes.byref(h)))
        self.handle, self.n_ref, self.p, self.n = h, nr, int(p), int(g.n)

    def edges(self):
        e = np.empty((self.n_ref, self.p + 1), dtype=np.int32)
        check(_lib().rfd_subband_edges(self.handle, e.ctypes.data_as(ctypes.c_void_p)))
        return e

    def filter_reference(self, dtilde, psd, href, halo, out=None, stream=None):
        ld = qref_ld(self.n, halo)
        if out is None:
            out = torch.zeros((self.n_ref, self.p, ld), dtype=torch.complex64, device="cuda")
        check(_lib().rfd_subband_filter_reference(self.handle, _ptr(dtilde), _ptr(psd), _ptr(href), int(halo),
                                                  _ptr(out), _stream(stream)))
        return out

    def shares(self, psd, taps, k, lag, ref_of, stream=None):
        ro, rop = _i32_host(ref_of)
        u = torch.zeros((len(ro), self.p), dtype=torch.float32, device="cuda")
        check(_lib().rfd_subband_shares(self.handle, _ptr(psd), _ptr(taps), int(taps.shape[-1]), _ptr(k), _ptr(lag),
                                        rop, len(ro), _ptr(u), _stream(stream)))
        return u

    def chi2(self, qband, halo, taps, k, lag, sigma, u, ref_of, trig, n_trig, zb=False, stream=None):
        ro, rop = _i32_host(ref_of)
        c = torch.zeros(max(int(n_trig), 1), dtype=torch.float32, device="cuda")
        z = torch.zeros((max(int(n_trig), 1), self.p), dtype=torch.complex64, device="cuda") if zb else None
        check(_lib().rfd_subband_chi2(self.handle, _ptr(qband), int(halo), _ptr(taps), int(taps.shape[-1]), _ptr(k),
                                      _ptr(lag), _ptr(sigma), _ptr(u), rop, len(ro), _ptr(trig), int(n_trig), _ptr(c),
                                      _ptr(z), _stream(stream)))
        return (c[:n_trig], z[:n_trig] if zb else None)

    def close(self):
        if self.handle:
            _lib().rfd_subband_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

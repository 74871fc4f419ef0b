"""Autotuner for the tensor-core ratio filter: picks the plan's tile choices by timing them.

The choices (rfd_plan_options): templates per tile for each K class, whether a tile may mix
templates of different K (padding the short ones) or must split where K changes, the number
of persistent CTAs, above which K templates go to the long-tap kernel (templates on the
MMA's M side, time on its N side), and above which K they go to the block-FFT kernel (FP32
overlap-save transforms on the CUDA cores, cheaper than the contraction for long taps), and
how small a reference's last long-kernel tile may be before its templates go to the block-FFT
kernel instead of padding a 64-template tile.  Each candidate plan is built through the C ABI,
given the bank's taps, and timed on the q_ref buffer with CUDA events after an L2 flush; the
fastest wins.  Results are cached
in a JSON file keyed by the workload's signature (grid, precision, the (reference, K)
histogram, the device), so a bank is tuned once.
"""
import hashlib
import json
import os

import numpy as np
import torch

from . import Plan, CANDIDATE_DTYPE

DEFAULT_CANDIDATES = [
    {"mix_k": 1},
    {"mix_k": 0},
    {"mix_k": 1, "tile_nt": [64, 64, 32]},
    {"mix_k": 0, "tile_nt": [64, 64, 32]},
    {"mix_k": 1, "long_k": 512},
    {"mix_k": 1, "long_k": 128},
    {"mix_k": 1, "long_k": 0},
    {"mix_k": 1, "fft_k": 256},
    {"mix_k": 1, "fft_k": 128},
    {"mix_k": 1, "fft_k": 0},
    {"mix_k": 1, "fft_k": 128, "long_k": 0},
    {"mix_k": 1, "fft_rem": 16},
    {"mix_k": 1, "fft_rem": 40},
    {"mix_k": 0, "fft_rem": 16},
]


def signature(g, precision, ref_of, k):
    ref_of = np.asarray(ref_of, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    pairs, counts = np.unique(np.stack([ref_of, (k + 15) // 16]), axis=1, return_counts=True)
    h = hashlib.sha256()
    h.update(repr((float(g.fs), int(g.n), float(g.f_low), int(g.pn_flags), int(precision))).encode())
    h.update(pairs.tobytes())
    h.update(counts.tobytes())
    h.update(torch.cuda.get_device_name().encode())
    return h.hexdigest()[:24]


def _time_plan(plan, qref, qscale, cand, cnt, reps, flush):
    for _ in range(2):
        plan.ratio_filter_batch(qref, qscale, cand, cnt)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.random_(0, 255)          # every timed call starts from a cold L2, as a search step does
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        plan.ratio_filter_batch(qref, qscale, cand, cnt)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def autotune(ctx, g, n_ref, ref_of, k, precision, window, threshold, halo, taps, k_stride, lag, sigma,
             qref, qscale, cache_path=None, candidates=None, reps=3):
    """Returns (options, report): the fastest candidate's options and every candidate's time (ms).
    The cache key covers the workload, the candidate list and the library version, so a cached
    choice is never reused for a different set of choices or kernels."""
    from . import _native
    cands = candidates or DEFAULT_CANDIDATES
    sig = signature(g, precision, ref_of, k) + "-" + hashlib.sha256(
        (json.dumps(cands, sort_keys=True) + str(_native.load().rfd_version())).encode()).hexdigest()[:8]
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if sig in cache:
            return cache[sig]["options"], cache[sig]
    cand = torch.zeros((1 << 22) * CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")     # larger than the 126 MB L2
    report = []
    for opts in cands:
        plan = Plan(ctx, g, n_ref, ref_of, k, precision, window, threshold, halo, options=opts)
        plan.set_taps(taps, k_stride, lag, sigma)
        ms = _time_plan(plan, qref, qscale, cand, cnt, reps, flush)
        report.append({"options": opts, "ms": ms, "executed_tflop": plan.executed_flops() / 1e12})
        plan.close()
    best = min(report, key=lambda r: r["ms"])
    entry = {"options": best["options"], "ms": best["ms"], "candidates": report}
    if cache_path:
        cache[sig] = entry
        d = os.path.dirname(os.path.abspath(cache_path))
        os.makedirs(d, exist_ok=True)
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return best["options"], entry

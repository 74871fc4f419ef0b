"""Oracle side of the learned-tap tests: exact taps at a fixed lag (the networks' training
targets), the templates' own lags, the references' autocorrelations and the network inputs.

Calls only oracle/ and workload/.  The per-template work (ratio spectrum, radix-2 inverse FFT,
lag search) runs in a spawn-started process pool so that a few thousand targets take seconds.
"""
import multiprocessing as mp
import os
import sys

import numpy as np

from oracle import mlp, ratio, waveform as wf


def _one(args):
    fs, n, f_low, pn, p, ref, K, alpha, lag, want_own = args
    g = ratio.impulse_response(ratio.ratio_spectrum(fs, n, f_low, p, ref, pn))
    own = ratio.choose_lag(ratio.window_energy(g, ratio.tukey(K, alpha)), K) if want_own else 0
    taps = ratio.taps_at_lag(g, K, alpha, lag) if lag is not None else None
    return own, taps


def _spawn_ok():
    """A spawned worker re-imports the parent's main module: it needs a file or a module name."""
    main = sys.modules.get("__main__")
    spec = getattr(main, "__spec__", None)
    path = getattr(main, "__file__", None)
    return spec is not None or (path is not None and os.path.exists(path))


def _map(jobs, procs):
    if procs is None:
        procs = min(16, os.cpu_count() or 1)
    if procs <= 1 or len(jobs) < 16 or not _spawn_ok():
        return [_one(j) for j in jobs]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_one, jobs, chunksize=max(1, len(jobs) // (4 * procs)))


def own_lags(fs, n, f_low, pn, params, ref_params, ref_of, K=128, alpha=0.1, procs=None):
    jobs = [(fs, n, f_low, pn, p, ref_params[r], K, alpha, None, True) for p, r in zip(params, ref_of)]
    return np.array([o for o, _ in _map(jobs, procs)], dtype=np.int64)


def targets(fs, n, f_low, pn, params, ref_params, ref_of, lag_of_ref, K=128, alpha=0.1, procs=None):
    """Exact taps rho[k] = w[k] g[(s_r + k) mod n] of every template at its reference's lag."""
    jobs = [(fs, n, f_low, pn, p, ref_params[r], K, alpha, int(lag_of_ref[r]), False)
            for p, r in zip(params, ref_of)]
    return np.stack([t for _, t in _map(jobs, procs)])


def autocorr(fs, n, f_low, pn, ref_params, psd, K=128):
    out = []
    for r in ref_params:
        h = wf.template(fs, n, f_low, r, pn)
        out.append(ratio.autocorrelation(h, psd, fs / n, n, K - 1))
    return np.stack(out)


def inputs(fs, f_low, pn, params, ref_params, ref_of, mu, sd):
    """Network inputs (n, 20) of every template under its own network's standardisation."""
    out = np.empty((len(params), mlp.N_FEAT))
    for r in range(len(ref_params)):
        sel = np.nonzero(ref_of == r)[0]
        if len(sel):
            out[sel] = mlp.network_inputs(params[sel], ref_params[r], mu[r], sd[r], fs, f_low, pn)
    return out


def init_weights(n_nets, seed):
    """Per network W ~ U(-1/sqrt(in), 1/sqrt(in)), b likewise, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    flat = []
    for _ in range(n_nets):
        parts = []
        for (o, i) in mlp.init_shapes():
            lim = 1.0 / np.sqrt(i)
            parts.append(rng.uniform(-lim, lim, (o, i)).ravel())
            parts.append(rng.uniform(-lim, lim, o))
        flat.append(np.concatenate(parts))
    return np.stack(flat).astype(np.float32)


def unflatten(w):
    """Flat per-network weights -> (W list, b list) in FP64."""
    W, b, off = [], [], 0
    for (o, i) in mlp.init_shapes():
        W.append(np.asarray(w[off:off + o * i], dtype=np.float64).reshape(o, i))
        off += o * i
        b.append(np.asarray(w[off:off + o], dtype=np.float64))
        off += o
    return W, b


def flatten(W, b):
    return np.concatenate([np.concatenate([x.ravel(), y.ravel()]) for x, y in zip(W, b)])

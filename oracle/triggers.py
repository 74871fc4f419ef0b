"""|z|^2 threshold crossings and per-window maxima (oracle; test infrastructure).

Table II's last two stages, "peak find" and "trigger accumulation": the SNR series is
reduced to one candidate per time window.  Window w holds the true sample indices
t in [w W, (w+1) W) (the last window is partial when W does not divide N).  In each
window the peak p* = max_t |z[t]|^2 is taken (ties to the smallest t) and a trigger
(w, t*, p*, z[t*]) is emitted when p* > threshold (strict).
"""
import numpy as np


def window_triggers(z, W, thr, tol=None):
    """Triggers of one template's series, sorted by window.  With `tol`, each trigger also
    reports whether the window is ambiguous under a relative error budget tol: its peak lies
    within 4 tol of the threshold, or its runner-up within 4 tol of the peak."""
    z = np.asarray(z)
    n = len(z)
    p = np.abs(z) ** 2
    nw = (n + W - 1) // W
    pad = np.full(nw * W, -np.inf)
    pad[:n] = p
    blocks = pad.reshape(nw, W)
    arg = np.argmax(blocks, axis=1)                 # first maximum = smallest t
    peak = blocks[np.arange(nw), arg]
    out = []
    for w in np.nonzero(peak > thr)[0]:
        t = int(w * W + arg[w])
        rec = {"w": int(w), "t": t, "p": float(peak[w]), "z": complex(z[t])}
        out.append(rec)
    if tol is not None:
        amb = []
        for w in range(nw):
            row = blocks[w]
            pk = peak[w]
            near_thr = abs(pk - thr) <= 4.0 * tol * thr
            if pk > thr or near_thr:
                second = np.max(np.delete(row, arg[w])) if W > 1 else -np.inf
                near_peak = (pk - second) <= 4.0 * tol * pk
                if near_thr or near_peak:
                    amb.append(int(w))
        return out, amb
    return out


def window_triggers_bruteforce(z, W, thr):
    """Plain loop version of window_triggers, for tiny inputs."""
    out = []
    n = len(z)
    w = 0
    while w * W < n:
        best_t, best_p = None, None
        for t in range(w * W, min((w + 1) * W, n)):
            pv = z[t].real ** 2 + z[t].imag ** 2
            if best_p is None or pv > best_p:
                best_t, best_p = t, pv
        if best_p > thr:
            out.append({"w": w, "t": best_t, "p": best_p, "z": complex(z[best_t])})
        w += 1
    return out

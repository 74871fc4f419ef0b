"""Chi^2-fitted ratio taps with an L2 ridge (Sec. V.A, Eq. 4), in FP64 (oracle; test
infrastructure).

Sec. V.A builds the taps by fitting their frequency response to the ratio, weighted toward the
detector's sensitive band, adds a ridge penalty on the taps (Hoerl & Kennard) so that the fit
stays well behaved where the weight is small, and tunes the number of taps to a target match.
Written in this implementation's conventions (the taps act on the reference series and model
conj(R), the Eq. 3 conjugation reading): taps rho placed at lag s have the response

  A_k = sum_n rho_n exp(-2 pi i k (s + n) / N),

and are fitted to G_k = conj(h_j,k / h_r,k) on the reference band with the reference's SNR
density as the weight (the data reach the ratio filter already band-passed by the reference):

  chi^2(rho) = sum_k w_k |G_k - A_k|^2 + lam |rho|^2,   w_k = 4 df |h_r,k|^2 / S_k,
  lam = eps C_r[0].

Its minimiser solves the Hermitian Toeplitz normal equations

  sum_m (C_r[n - m] + lam delta_nm) rho_m = b_n,   b_n = sum_k w_k G_k exp(+2 pi i k (s + n) / N),

with C_r the reference autocorrelation of Eq. 6.  The same quantities give the match of the
fitted taps to the template, |rho^H b| / sqrt(rho^H C_r rho  sigma_j^2), sigma_j^2 = 4 df sum
|h_j|^2 / S.  The lag is placed by the window-energy rule of ratio.place_taps (the same lag the
windowed taps use).  This module solves the system with a dense library solve.
"""
import math

import numpy as np

from . import ratio as _ratio
from . import waveform as _wf


def weights(h_ref, psd, df):
    """w_k = 4 df |h_r,k|^2 / S_k on the reference's non-zero bins (k <= N/2), else 0."""
    w = np.zeros(len(h_ref))
    nz = np.nonzero(h_ref)[0]
    w[nz] = 4.0 * df * np.abs(h_ref[nz]) ** 2 / psd[nz]
    return w


def rhs(G, w, s, K):
    """b_n = sum_k w_k G_k exp(+2 pi i k (s + n) / N), n < K (one inverse transform of w G)."""
    n = len(G)
    wg = np.zeros(n, dtype=np.complex128)
    wg[: len(w)] = w * G[: len(w)]
    full = _ratio.impulse_response(wg) * n
    return full[(s + np.arange(K)) % n]


def toeplitz(C, K):
    """T[n, m] = C[n - m] from C[l], l = -(K-1) .. K-1 stored at index l + K - 1."""
    mid = (len(C) - 1) // 2
    i = np.arange(K)
    return C[mid + i[:, None] - i[None, :]]


def solve(C, b, eps):
    """The ridge-regularised normal equations, by a dense solve."""
    K = len(b)
    mid = (len(C) - 1) // 2
    T = toeplitz(C, K) + eps * C[mid].real * np.eye(K)
    return np.linalg.solve(T, b)


def fit_match(rho, b, C, sigma_j_sq):
    """|rho^H b| / sqrt(rho^H C rho sigma_j^2): the match of the fitted taps to the template."""
    T = toeplitz(C, len(rho))
    s_eff = float(np.real(np.conj(rho) @ (T @ rho)))
    return abs(np.vdot(rho, b)) / math.sqrt(s_eff * sigma_j_sq), s_eff


def design(fs, n, f_low, tmpl_params, ref_params, psd, K, eps=1e-6, alpha=0.1, pn_flags=0):
    """Fitted taps, lag, sigma_eff and match for one template at a given K."""
    df = fs / n
    G = _ratio.ratio_spectrum(fs, n, f_low, tmpl_params, ref_params, pn_flags)
    g = _ratio.impulse_response(G)
    s = _ratio.choose_lag(_ratio.window_energy(g, _ratio.tukey(K, alpha)), K)
    h_ref = _wf.template(fs, n, f_low, ref_params, pn_flags)
    h_j = _wf.template(fs, n, f_low, tmpl_params, pn_flags)
    w = weights(h_ref, psd, df)
    C = _ratio.autocorrelation(h_ref, psd, df, n, K - 1)
    b = rhs(G, w, s, K)
    rho = solve(C, b, eps)
    nz = np.nonzero(h_j)[0]
    sig_j2 = 4.0 * df * float(np.sum(np.abs(h_j[nz]) ** 2 / psd[nz]))
    m, s_eff = fit_match(rho, b, C, sig_j2)
    return {"lag": s, "taps": rho, "sigma_eff": math.sqrt(s_eff), "match": m, "b": b, "C": C,
            "sigma_j_sq": sig_j2}


def design_dynamic(fs, n, f_low, tmpl_params, ref_params, psd, buckets, target, eps=1e-6, alpha=0.1,
                   pn_flags=0):
    """The smallest bucket whose fitted taps reach the target match (else the largest bucket)."""
    out = None
    for K in sorted(buckets):
        out = design(fs, n, f_low, tmpl_params, ref_params, psd, K, eps, alpha, pn_flags)
        out["K"] = K
        if out["match"] >= target:
            break
    return out

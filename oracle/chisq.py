"""Sub-band chi^2 signal-consistency test through the ratio filter, in FP64 (oracle; test
infrastructure).

The paper's signal-consistency section (Sec. VI) notes that the time-frequency chi^2 test
(Allen 2005) splits the band into pieces and checks that the SNR accumulates in proportion, and
that the ratio filter extends to it: a template's sub-band SNR series is the ratio FIR applied
to the reference's sub-band series, so the data are filtered per sub-band once per reference.

Definitions (n samples, df = fs / n):
  w_k   = 4 df |h_r,k|^2 / S_k on the reference's band (its SNR density).
  edges e_0 = k_lo < e_1 < ... < e_p = k_hi + 1, e_b the first bin at which the running sum of
        w (in k order, from k_lo) reaches b W / p, W = sum w: p sub-bands of equal reference SNR.
  q_r,b[m] = sum_{k in band b} 4 df d_k conj(h_r,k) / S_k exp(+2 pi i k m / n)
        (sum_b q_r,b = q_r, the reference series of Eq. 1).
  z_b(t) = (1 / sigma_eff) sum_k rho[k] q_r,b[(t - s - k) mod n]       (Eq. 3 per sub-band)
  z(t)  = sum_b z_b(t)                                                  (the template's SNR)
  C_b[l] = sum_{k in band b} w_k exp(+2 pi i k l / n);  sigma_b^2 = rho^H C_b rho,
  u_b   = sigma_b^2 / sigma_eff^2 (sum_b u_b = 1): the share of the effective template's power.
  chi^2(t) = sum_b |z_b(t) - u_b z(t)|^2 / u_b,
which in Gaussian noise follows a chi^2 distribution with 2 (p - 1) degrees of freedom, and for
a signal that matches the effective template has the same distribution (no excess).
"""
import numpy as np

from . import fft as _fft
from . import ratio as _ratio


def band_weights(h_ref, psd, df):
    w = np.zeros(len(h_ref))
    nz = np.nonzero(h_ref)[0]
    w[nz] = 4.0 * df * np.abs(h_ref[nz]) ** 2 / psd[nz]
    return w


def band_edges(h_ref, psd, df, p):
    """p sub-bands of equal reference SNR: e_b = first bin where the running sum reaches b W / p."""
    w = band_weights(h_ref, psd, df)
    nz = np.nonzero(w)[0]
    k_lo, k_hi = int(nz[0]), int(nz[-1])
    run = np.cumsum(w[k_lo:k_hi + 1])            # run[i] = sum of w over k_lo .. k_lo + i
    W = run[-1]
    edges = [k_lo]
    for b in range(1, p):
        i = int(np.argmax(run >= b * W / p))     # first i with run[i] >= b W / p
        edges.append(k_lo + i + 1)               # band b - 1 ends after bin k_lo + i
    edges.append(k_hi + 1)
    return np.array(edges, dtype=np.int64)


def band_series(dtilde, h_ref, psd, df, n, edges):
    """q_r,b for each sub-band (unnormalised inverse transforms of the band-limited spectra)."""
    out = []
    for b in range(len(edges) - 1):
        c = np.zeros(n, dtype=np.complex128)
        k = np.arange(edges[b], edges[b + 1])
        c[k] = 4.0 * df * dtilde[k] * np.conj(h_ref[k]) / psd[k]
        out.append(_fft.ifft(c))
    return np.stack(out)


def band_autocorr(h_ref, psd, df, n, edges, max_lag):
    """C_b[l], l = -max_lag .. max_lag, for each sub-band."""
    w = band_weights(h_ref, psd, df)
    lags = np.arange(-max_lag, max_lag + 1)
    out = []
    for b in range(len(edges) - 1):
        k = np.arange(edges[b], edges[b + 1])
        ph = np.exp(2j * np.pi * np.outer(lags, k) / n)
        out.append(ph @ w[k])
    return np.stack(out)


def subband_chi2(q_bands, rho, s, sigma_eff, C_bands, t):
    """chi^2 and the sub-band SNRs z_b at the samples t (array)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.int64))
    p = q_bands.shape[0]
    zb = np.stack([_ratio.ratio_fir_at(q_bands[b], rho, s, t) / sigma_eff for b in range(p)])   # [p][len(t)]
    z = zb.sum(axis=0)
    K = len(rho)
    mid = (C_bands.shape[1] - 1) // 2
    i = np.arange(K)
    u = np.empty(p)
    for b in range(p):
        T = C_bands[b][mid + i[:, None] - i[None, :]]       # T[n, m] = C_b[n - m]
        u[b] = float(np.real(np.conj(rho) @ (T @ rho))) / sigma_eff ** 2
    chi2 = np.sum(np.abs(zb - u[:, None] * z[None, :]) ** 2 / u[:, None], axis=0)
    return chi2, zb, u

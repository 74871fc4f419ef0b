"""Ratio-filter dechirping in FP64 (oracle; test infrastructure).

Eq. 2 writes a target template as h = h_ref * (h / h_ref).  Substituting into Eq. 1 gives
Eq. 3: the target's SNR series is the reference's series convolved with the inverse
transform of the ratio.  Because Eq. 1 correlates with conj(h), the kernel that acts on the
reference series is the inverse transform of conj(R), R = h / h_ref (the Eq. 3 conjugation
reading; the K = N identity test pins it).  Sec. V: the kernel is short because the ratio
varies slowly; it is cut to K taps.  The cut used here is the windowed, truncated inverse
transform: a Tukey window placed where it captures the most window-weighted energy.

Discrete definitions (n samples, df = fs/n, band B_r = [k_lo, k_hi_ref] of the reference):

  G[k]   = exp(+i (Psi_j(f_k) - Psi_r(f_k)))   for k in B_r up to the template's own cutoff
         = 0                                   for k in B_r above the template's cutoff
         = linear fill on the out-of-band arc (magnitude and shortest-arc phase,
           from G[k_hi_ref] round to G[k_lo])
  g[n]   = (1/N) sum_k G[k] exp(+2 pi i k n / N)
  E[s]   = sum_{k<K} w[k]^2 |g[(s+k) mod N]|^2,      s in [-N/2, N/2)
  s_j    = argmax E (values within 1e-9 relative of the maximum tie; ties go to the
           placement closest to s = -K/2, then to the smaller s)
  rho[k] = w[k] g[(s_j + k) mod N]
  qhat[m] = sum_{k<K} rho[k] q_r[(m - s_j - k) mod N]                      (Eq. 3)
  sigma_eff^2 = sum_{n,n'} rho[n] conj(rho[n']) C_r[n' - n]                (Eqs. 5-6)
  C_r[l] = 4 df sum_{k in B_r} |h_r,k|^2 / S_k exp(+2 pi i k l / N)
  z[m]   = qhat[m] / sigma_eff
"""
import math

import numpy as np

from . import fft as _fft
from . import waveform as _wf


# ---------------------------------------------------------------- ratio spectrum (Eq. 2)
def fill_out_of_band(G, k_lo, k_hi):
    """Fill the arc k_hi+1 .. N-1, 0 .. k_lo-1 by linear interpolation of magnitude and of
    phase (shortest arc) from G[k_hi] to G[k_lo].  Only the in-band values matter to the
    filter (Sec. V.A); the fill keeps the ratio smooth round the circle so that its
    inverse transform stays short, and makes G == 1 when template == reference."""
    n = len(G)
    L = n - (k_hi - k_lo + 1)
    if L <= 0:
        return G
    a, b = G[k_hi], G[k_lo]
    ma, mb = abs(a), abs(b)
    pa, pb = math.atan2(a.imag, a.real), math.atan2(b.imag, b.real)
    dp = pb - pa
    dp -= 2.0 * math.pi * math.floor((dp + math.pi) / (2.0 * math.pi))  # into [-pi, pi)
    i = np.arange(1, L + 1, dtype=np.float64)
    s = i / (L + 1)
    vals = ((1.0 - s) * ma + s * mb) * np.exp(1j * (pa + s * dp))
    idx = (k_hi + i.astype(np.int64)) % n
    G[idx] = vals
    return G


def ratio_spectrum(fs, n, f_low, tmpl_params, ref_params, pn_flags=0):
    """conj(h_j / h_r) on the full circle k = 0..N-1 (Eq. 2 conjugated, with the fill).
    The phase difference is formed from the two FP64 phases, never by dividing complex
    numbers, and the amplitude ratio is 1 where both templates are non-zero."""
    m1, m2, c1, c2, lam = [float(x) for x in tmpl_params]
    r1, r2, rc1, rc2, rlam = [float(x) for x in ref_params]
    k_lo, k_hi = _wf.band(fs, n, f_low, r1, r2)
    _, k_hi_t = _wf.band(fs, n, f_low, m1, m2)
    G = np.zeros(n, dtype=np.complex128)
    k_top = min(k_hi, k_hi_t)
    if k_top >= k_lo:
        f = np.arange(k_lo, k_top + 1, dtype=np.float64) * (fs / n)
        dpsi = (_wf.phase(f, m1, m2, c1, c2, lam, pn_flags)
                - _wf.phase(f, r1, r2, rc1, rc2, rlam, pn_flags))
        G[k_lo:k_top + 1] = np.exp(1j * dpsi)
    return fill_out_of_band(G, k_lo, k_hi)


def impulse_response(G):
    """g = (1/N) IDFT_N(G): the exact (untruncated) ratio kernel r(t) of Sec. III."""
    return _fft.ifft(G) / len(G)


# ---------------------------------------------------------------- taps (Sec. V)
def tukey(K, alpha):
    """Symmetric Tukey window of length K (flat top, cosine tapers of alpha (K-1)/2)."""
    if K == 1:
        return np.ones(1)
    n = np.arange(K, dtype=np.float64)
    w = np.ones(K)
    if alpha <= 0:
        return w
    if alpha >= 1:
        return 0.5 * (1.0 - np.cos(2.0 * math.pi * n / (K - 1)))
    width = alpha * (K - 1) / 2.0
    lo = n < width
    w[lo] = 0.5 * (1.0 + np.cos(math.pi * (n[lo] / width - 1.0)))
    hi = n > (K - 1) - width
    w[hi] = 0.5 * (1.0 + np.cos(math.pi * (n[hi] / width - 2.0 / alpha + 1.0)))
    return w


def window_energy(g, w):
    """E[s] for s = -N/2 .. N/2-1 (returned in that order)."""
    n = len(g)
    e = np.abs(g) ** 2
    E = np.zeros(n)
    for k in range(len(w)):
        E += w[k] ** 2 * np.roll(e, -k)   # E[m] += w[k]^2 e[(m+k) mod N]
    return np.concatenate([E[n // 2:], E[:n // 2]])


LAG_TIE_RTOL = 1e-9


def choose_lag(E, K):
    """Maximiser of the window energy with the tie rule stated in the module docstring."""
    n = len(E)
    s = np.arange(-n // 2, n // 2)
    emax = E.max()
    cand = s[E >= emax * (1.0 - LAG_TIE_RTOL)]
    d = np.abs(cand + K // 2)
    best = cand[d == d.min()]
    return int(best.min())


def taps_at_lag(g, K, alpha, s):
    """Windowed taps placed at a given lag: rho[k] = w[k] g[(s+k) mod N]."""
    n = len(g)
    return tukey(K, alpha) * g[(s + np.arange(K)) % n]


def place_taps(g, K, alpha):
    """(s_j, rho_j): lag and windowed taps rho[k] = w[k] g[(s+k) mod N]."""
    w = tukey(K, alpha)
    s = choose_lag(window_energy(g, w), K)
    return s, taps_at_lag(g, K, alpha, s)


# ---------------------------------------------------------------- the FIR of Eq. 3
def ratio_fir(q_ref, rho, s):
    """Direct circular sum qhat[m] = sum_k rho[k] q_ref[(m - s - k) mod N] (no FFT, so it is
    independent of the matched-filter code path)."""
    out = np.zeros(len(q_ref), dtype=np.complex128)
    for k in range(len(rho)):
        out += rho[k] * np.roll(q_ref, s + k)   # roll(q, a)[m] = q[m - a]
    return out


def ratio_fir_at(q_ref, rho, s, t):
    """qhat at the sample indices t only (for spot checks at full size)."""
    n = len(q_ref)
    t = np.asarray(t, dtype=np.int64)
    k = np.arange(len(rho))
    idx = (t[:, None] - s - k[None, :]) % n
    return (q_ref[idx] * rho[None, :]).sum(axis=1)


# ---------------------------------------------------------------- normalisation (Eqs. 5-6)
def autocorrelation(h_ref, psd, df, n, max_lag):
    """C_r[l] for l = -max_lag .. max_lag (index l + max_lag): the reference's
    autocorrelation (h_ref|h_ref)(t) of Eq. 6 on the sample grid,
    C_r[l] = sum_k w_k exp(+2 pi i k l / n), w_k = 4 df |h_ref,k|^2 / S_k, which is n times
    the inverse DFT of w at l (numpy's FFT as the library step)."""
    w = np.zeros(n, dtype=np.complex128)
    nz = np.nonzero(h_ref)[0]
    w[nz] = 4.0 * df * np.abs(h_ref[nz]) ** 2 / psd[nz]
    full = np.fft.ifft(w) * n
    lags = np.arange(-max_lag, max_lag + 1)
    return full[lags % n]


def sigma_eff_sq_parseval(rho, C):
    """Eq. 6 collapsed to the taps: sum_{n,n'} rho[n] conj(rho[n']) C[n' - n]."""
    K = len(rho)
    mid = (len(C) - 1) // 2
    i = np.arange(K)
    Cmat = C[mid + i[None, :] - i[:, None]]          # Cmat[n, n'] = C[n' - n]
    return float(np.real(rho @ Cmat @ np.conj(rho)))


def effective_response(rho, s, n):
    """A[k] = sum_n rho[n] exp(-2 pi i k (s + n) / N) for k = 0..N-1: the frequency response
    of the placed taps; h_eff = h_ref conj(A)."""
    buf = np.zeros(n, dtype=np.complex128)
    buf[(s + np.arange(len(rho))) % n] = rho
    return _fft.fft(buf)


def sigma_eff_sq_freq(rho, s, h_ref, psd, df, n):
    """Eq. 5: 4 df sum_k |h_ref,k|^2 / S_k |A_k|^2 (frequency-domain form)."""
    A = effective_response(rho, s, n)[: n // 2 + 1]
    nz = np.nonzero(h_ref)[0]
    return 4.0 * df * float(np.sum(np.abs(h_ref[nz]) ** 2 / psd[nz] * np.abs(A[nz]) ** 2))


def tap_match(h_j, rho, s, h_ref, psd, df, n):
    """Phase-maximised overlap of the exact template with the tap-reconstructed template
    h_eff = h_ref conj(A) (Sec. V.A's target match), at the fixed lag."""
    A = effective_response(rho, s, n)[: n // 2 + 1]
    h_eff = h_ref * np.conj(A)
    nz = np.nonzero(psd)[0]
    inner = 4.0 * df * np.sum(np.conj(h_j[nz]) * h_eff[nz] / psd[nz])
    sj = 4.0 * df * np.sum(np.abs(h_j[nz]) ** 2 / psd[nz])
    se = 4.0 * df * np.sum(np.abs(h_eff[nz]) ** 2 / psd[nz])
    return float(abs(inner) / math.sqrt(sj * se))


# ---------------------------------------------------------------- tap count (Sec. V.A)
def energy_span(g, frac=0.999):
    """Shortest circular span holding `frac` of sum |g|^2."""
    e = np.abs(g) ** 2
    n = len(e)
    total = e.sum()
    c = np.concatenate([[0.0], np.cumsum(np.concatenate([e, e]))])
    lo, hi = 1, n
    while lo < hi:
        L = (lo + hi) // 2
        best = np.max(c[L:L + n] - c[:n])
        if best >= frac * total:
            hi = L
        else:
            lo = L + 1
    return lo


def k_bucket(g, buckets, frac=0.999):
    span = energy_span(g, frac)
    for b in sorted(buckets):
        if b >= span:
            return b
    return max(buckets)


# ---------------------------------------------------------------- one template, end to end
def design(fs, n, f_low, tmpl_params, ref_params, psd, K, alpha=0.1, pn_flags=0,
           with_match=True):
    """Taps, lag, sigma_eff and match for one template against its reference."""
    df = fs / n
    G = ratio_spectrum(fs, n, f_low, tmpl_params, ref_params, pn_flags)
    g = impulse_response(G)
    s, rho = place_taps(g, K, alpha)
    h_ref = _wf.template(fs, n, f_low, ref_params, pn_flags)
    C = autocorrelation(h_ref, psd, df, n, K - 1)
    sig2 = sigma_eff_sq_parseval(rho, C)
    out = {"lag": s, "taps": rho, "sigma_eff": math.sqrt(sig2), "g": g}
    if with_match:
        h_j = _wf.template(fs, n, f_low, tmpl_params, pn_flags)
        out["match"] = tap_match(h_j, rho, s, h_ref, psd, df, n)
    return out


def snr_series(q_ref, taps, lag, sigma_eff):
    """z_j[m] = qhat_j[m] / sigma_eff,j."""
    return ratio_fir(q_ref, taps, lag) / sigma_eff

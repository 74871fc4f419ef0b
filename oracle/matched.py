"""FINDCHIRP matched filter, Eq. 1 discretised (oracle; test infrastructure).

Eq. 1: (s|h)(t) = 4 int_0^inf s(f) h*(f) / S_n(f) exp(2 pi i f t) df.  On the grid
f_k = k df, t_m = m / fs this is

  c[k] = 4 df d[k] conj(h[k]) / S[k]   for k in the band, 0 for every other k in [0, N)
  q[m] = sum_{k=0}^{N-1} c[k] exp(+2 pi i k m / N)          (unnormalised inverse FFT)
  z[m] = q[m] / sigma(h),  sigma^2 = (h|h) = 4 df sum_k |h[k]|^2 / S[k]

which is the point-wise multiply + inverse FFT described in Sec. III.  With noise bins
sqrt(S/(4 df)) (a + i b), a, b ~ N(0,1), z is a complex SNR with E|z|^2 = 2.
"""
import numpy as np

from . import fft as _fft


def sigma_sq(h, psd, df):
    """(h|h) = 4 df sum_k |h_k|^2 / S_k over the bins where h is non-zero (Eq. 5 with R = 1)."""
    h = np.asarray(h)
    nz = h != 0
    return 4.0 * df * float(np.sum(np.abs(h[nz]) ** 2 / psd[nz]))


def weighted_spectrum(dtilde, h, psd, df, n):
    """c[k] of the discretised Eq. 1, length n (the upper half k > n/2 is zero)."""
    c = np.zeros(n, dtype=np.complex128)
    h = np.asarray(h, dtype=np.complex128)
    nz = np.nonzero(h)[0]
    c[nz] = 4.0 * df * np.asarray(dtilde)[nz] * np.conj(h[nz]) / psd[nz]
    return c


def filter_unnormalised(dtilde, h, psd, df, n):
    """q[m] = sum_k c[k] exp(+2 pi i k m / N): the reference SNR series of Eq. 3 before
    normalisation ((s|h)_ref in the paper's notation)."""
    return _fft.ifft(weighted_spectrum(dtilde, h, psd, df, n))


def findchirp(dtilde, h, psd, df, n):
    """Normalised complex SNR series z[m] = q[m] / sigma(h) (Eq. 1)."""
    return filter_unnormalised(dtilde, h, psd, df, n) / np.sqrt(sigma_sq(h, psd, df))

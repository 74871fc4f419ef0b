"""Hand-written iterative radix-2 FFT in complex128 (oracle; test infrastructure).

The matched filter of Eq. 1 is evaluated, as in FINDCHIRP (Sec. III), by a pointwise
product followed by an inverse FFT.  This is the textbook Cooley-Tukey decimation-in-time
algorithm: bit-reversal permutation, then log2(N) butterfly stages.  No normalisation is
applied in either direction: fft computes X[k] = sum_n x[n] exp(-2 pi i k n / N) and ifft
computes x[n] = sum_k X[k] exp(+2 pi i k n / N).
"""
import numpy as np


def _bit_reverse(n: int) -> np.ndarray:
    bits = n.bit_length() - 1
    idx = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((idx >> b) & 1) << (bits - 1 - b)
    return rev


def _transform(x, sign: float) -> np.ndarray:
    a = np.array(x, dtype=np.complex128)
    n = a.shape[-1]
    if n < 1 or (n & (n - 1)) != 0:
        raise ValueError("radix-2 FFT needs a power-of-two length")
    lead = a.shape[:-1]
    a = a[..., _bit_reverse(n)]
    m = 2
    while m <= n:
        half = m // 2
        w = np.exp(sign * 2j * np.pi * np.arange(half) / m)
        a = a.reshape(lead + (n // m, m))
        top = a[..., :half]
        bot = a[..., half:] * w
        a = np.concatenate([top + bot, top - bot], axis=-1)
        m *= 2
    return a.reshape(lead + (n,))


def fft(x) -> np.ndarray:
    """Unnormalised forward DFT, exp(-2 pi i k n / N)."""
    return _transform(x, -1.0)


def ifft(x) -> np.ndarray:
    """Unnormalised inverse DFT, exp(+2 pi i k n / N) (no 1/N)."""
    return _transform(x, +1.0)

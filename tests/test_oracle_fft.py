"""Pins for the oracle's radix-2 FFT: brute-force DFT, round trip, Parseval, closed forms."""
import numpy as np
import pytest

from oracle import fft


def brute_dft(x, sign):
    n = len(x)
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n) @ x


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256])
def test_fft_matches_bruteforce_dft(n, rng):
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for f, sign in ((fft.fft, -1.0), (fft.ifft, +1.0)):
        ref = brute_dft(x, sign)
        assert np.max(np.abs(f(x) - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_round_trip_and_parseval(rng):
    n = 4096
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = fft.fft(x)
    assert np.max(np.abs(fft.ifft(X) / n - x)) < 1e-13
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(X) ** 2) / n) < 1e-10 * np.sum(np.abs(x) ** 2)


def test_closed_forms():
    n = 1024
    d = np.zeros(n, complex)
    d[0] = 1.0
    assert np.max(np.abs(fft.fft(d) - 1.0)) < 1e-15
    k0 = 37
    e = np.exp(2j * np.pi * k0 * np.arange(n) / n)
    X = fft.fft(e)
    ref = np.zeros(n, complex)
    ref[k0] = n
    assert np.max(np.abs(X - ref)) < 1e-9


def test_batched_rows_match_single(rng):
    x = rng.standard_normal((3, 64)) + 1j * rng.standard_normal((3, 64))
    Y = fft.ifft(x)
    for i in range(3):
        assert np.max(np.abs(Y[i] - fft.ifft(x[i]))) == 0.0


def test_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        fft.fft(np.zeros(12))

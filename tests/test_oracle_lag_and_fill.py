"""Pins of the oracle's tap placement (Sec. V: the window-energy lag and its tie rule, reading 6),
the tap count from the ratio's bandwidth (reading 15) and the out-of-band fill of the ratio
(reading 5), against brute force on tiny inputs, the exact maximisers for impulses and the fill's
invariants."""
import math

import numpy as np
import pytest

from oracle import ratio


def brute_window_energy(g, w):
    n = len(g)
    return {s: sum(w[k] ** 2 * abs(g[(s + k) % n]) ** 2 for k in range(len(w))) for s in range(-n // 2, n // 2)}


@pytest.mark.parametrize("n,K,alpha", [(64, 7, 0.1), (32, 12, 0.5), (16, 16, 1.0), (40, 1, 0.1)])
def test_window_energy_is_its_defining_sum(n, K, alpha):
    rng = np.random.default_rng(n * 100 + K)
    g = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    w = ratio.tukey(K, alpha)
    E = ratio.window_energy(g, w)
    ref = brute_window_energy(g, w)
    for s in range(-n // 2, n // 2):
        assert abs(E[s + n // 2] - ref[s]) <= 1e-12 * max(1.0, ref[s])


@pytest.mark.parametrize("n,K", [(256, 16), (256, 33), (1024, 64)])
def test_lag_for_a_single_impulse(n, K):
    """g = one impulse at p: the window-weighted energy is largest (and tied) exactly for the
    placements that put the impulse under the Tukey window's flat top, s = p - k for k in the
    flat top (wrapped into [-n/2, n/2)); the tie rule takes the one nearest -K/2, then the
    smaller.  The taps are then the impulse at k = p - s, unchanged by the flat top."""
    w = ratio.tukey(K, 0.1)
    flat = np.flatnonzero(w == w.max())
    for p in (0, 5, 40, n // 2 - 1, n // 2, n - 3, n - 40):
        g = np.zeros(n, complex)
        g[p] = 2.0 - 1.0j
        ties = sorted({(p - k + n // 2) % n - n // 2 for k in flat})
        want = min(ties, key=lambda x: (abs(x + K // 2), x))
        s, rho = ratio.place_taps(g, K, 0.1)
        assert s == want, (p, s, want)
        expect = np.zeros(K, complex)
        expect[(p - s) % n] = 2.0 - 1.0j
        assert np.array_equal(rho, expect)


def test_lag_tie_goes_to_the_placement_nearest_minus_half_k_then_the_smaller():
    """Two equal impulses whose flat-top placements exclude -K/2: the nearer set wins; when the
    two sets come equally near, the smaller placement wins."""
    n, K = 512, 16                                  # flat top k = 1 .. 14
    g = np.zeros(n, complex)
    g[40] = 1.0                                     # placements 26 .. 39: nearest 26, distance 34
    g[n - 40] = 1.0                                 # placements -54 .. -41: nearest -41, distance 33
    assert ratio.place_taps(g, K, 0.1)[0] == -41
    g = np.zeros(n, complex)
    g[30] = 1.0                                     # placements 16 .. 29: nearest 16, distance 24
    g[n - 31] = 1.0                                 # placements -45 .. -32: nearest -32, distance 24
    assert ratio.place_taps(g, K, 0.1)[0] == -32


@pytest.mark.parametrize("seed", range(4))
def test_lag_is_the_brute_force_maximiser(seed):
    rng = np.random.default_rng(100 + seed)
    n, K = 48, 9
    g = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    E = brute_window_energy(g, ratio.tukey(K, 0.1))
    best = max(E.values())
    ties = [s for s in E if E[s] >= best * (1 - 1e-9)]
    assert ratio.place_taps(g, K, 0.1)[0] == min(ties, key=lambda x: (abs(x + K // 2), x))


def brute_energy_span(g, frac):
    e = np.abs(g) ** 2
    n, total = len(e), e.sum()
    for L in range(1, n + 1):
        for a in range(n):
            if sum(e[(a + i) % n] for i in range(L)) >= frac * total:
                return L
    return n


@pytest.mark.parametrize("seed", range(6))
def test_energy_span_is_the_shortest_circular_window(seed):
    rng = np.random.default_rng(seed)
    n = 24
    g = rng.standard_normal(n) * np.exp(-0.5 * ((np.arange(n) - rng.integers(n)) / 3.0) ** 2) + 0j
    g = np.roll(g, rng.integers(n))
    for frac in (0.5, 0.9, 0.999):
        assert ratio.energy_span(g, frac) == brute_energy_span(g, frac), frac


def arc(G, k_lo, k_hi):
    """G[k_hi], the filled bins in circular order, G[k_lo]."""
    n = len(G)
    L = n - (k_hi - k_lo + 1)
    return np.array([G[(k_hi + i) % n] for i in range(L + 2)])


@pytest.mark.parametrize("pa,pb", [(0.3, 1.1), (3.0, -3.0), (-3.0, 3.0), (0.0, math.pi - 1e-9), (1.0, 1.0)])
def test_out_of_band_fill_invariants(pa, pb):
    """In-band values untouched; along the filled arc from G[k_hi] round to G[k_lo] the
    magnitude changes in equal steps and the phase turns by equal steps the short way round."""
    rng = np.random.default_rng(11)
    n, k_lo, k_hi = 64, 9, 40
    G = np.zeros(n, complex)
    G[k_lo:k_hi + 1] = rng.uniform(0.5, 2.0, k_hi - k_lo + 1) * np.exp(1j * rng.uniform(-3, 3, k_hi - k_lo + 1))
    G[k_hi] = 1.7 * np.exp(1j * pa)
    G[k_lo] = 0.4 * np.exp(1j * pb)
    band = G[k_lo:k_hi + 1].copy()
    out = ratio.fill_out_of_band(G.copy(), k_lo, k_hi)
    assert np.array_equal(out[k_lo:k_hi + 1], band)
    a = arc(out, k_lo, k_hi)
    steps = len(a) - 1
    mag = np.abs(a)
    assert np.max(np.abs(np.diff(mag, 2))) < 1e-12                 # linear in magnitude
    assert abs(mag[0] - 1.7) < 1e-15 and abs(mag[-1] - 0.4) < 1e-15
    turn = np.angle(a[1:] / a[:-1])                                  # each step's rotation
    assert np.max(np.abs(turn - turn[0])) < 1e-9                     # equal steps
    assert abs(turn[0] * steps) <= math.pi + 1e-9                    # the short way round
    total = (pb - pa + math.pi) % (2 * math.pi) - math.pi
    assert abs(turn[0] * steps - total) < 1e-9


def test_fill_of_a_unit_ratio_is_one():
    n, k_lo, k_hi = 128, 7, 60
    G = np.zeros(n, complex)
    G[k_lo:k_hi + 1] = 1.0
    assert np.array_equal(ratio.fill_out_of_band(G, k_lo, k_hi), np.ones(n, complex))

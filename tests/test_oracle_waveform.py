"""Pins for the oracle's TaylorF2 phase, using results derived independently of its code:

* (1/2pi) dPsi/df = t_c - tau(f), where tau is the post-Newtonian time to coalescence
  tau = 5 M / (256 eta v^8) [1 + (743/252 + 11 eta/3) v^2 - (32/5)(pi - beta/4) v^3]
  (Peters' chirp time at leading order, with the standard 1PN / 1.5PN corrections);
* the spin-orbit coefficient in its (chi_s, chi_a, delta) form,
  beta = (113/12 - 19 eta/3) chi_s + (113/12) delta chi_a;
* f_ISCO of a 1.4 + 1.4 Msun binary is about 1570 Hz.
"""
import math

import numpy as np
import pytest

from oracle import waveform as wf


def chirp_time(f, m1, m2, beta=0.0):
    M = (m1 + m2) * wf.T_SUN
    eta = m1 * m2 / (m1 + m2) ** 2
    v = (math.pi * M * f) ** (1.0 / 3.0)
    return 5.0 * M / (256.0 * eta * v ** 8) * (
        1.0 + (743.0 / 252.0 + 11.0 * eta / 3.0) * v ** 2 - 32.0 / 5.0 * (math.pi - beta / 4.0) * v ** 3)


@pytest.mark.parametrize("m1,m2,chi1,chi2", [(1.4, 1.4, 0, 0), (2.7, 1.1, 0, 0), (10.0, 3.0, 0.4, -0.3),
                                             (0.5, 0.2, 0.0, 0.0)])
def test_phase_derivative_is_chirp_time(m1, m2, chi1, chi2):
    flags = wf.PN_SO if (chi1 or chi2) else 0
    beta = wf.spin_orbit_beta(m1, m2, chi1, chi2) if flags else 0.0
    tc = 3.0
    for f in (20.0, 45.0, 100.0, 300.0):
        h = 1e-4 * f
        # fourth-order central difference
        d = (-wf.phase(f + 2 * h, m1, m2, chi1, chi2, 0, flags, tc) + 8 * wf.phase(f + h, m1, m2, chi1, chi2, 0, flags, tc)
             - 8 * wf.phase(f - h, m1, m2, chi1, chi2, 0, flags, tc) + wf.phase(f - 2 * h, m1, m2, chi1, chi2, 0, flags, tc)) / (12 * h)
        t = d / (2 * math.pi)
        ref = tc - chirp_time(f, m1, m2, beta)
        assert abs(t - ref) <= 1e-6 * max(1.0, abs(ref)), (f, t, ref)


def test_spin_orbit_alternative_form(rng):
    for _ in range(20):
        m1, m2 = sorted(rng.uniform(1, 20, 2))[::-1]
        c1, c2 = rng.uniform(-0.5, 0.5, 2)
        M = m1 + m2
        eta = m1 * m2 / M ** 2
        chis, chia, delta = 0.5 * (c1 + c2), 0.5 * (c1 - c2), (m1 - m2) / M
        alt = (113.0 / 12.0 - 19.0 * eta / 3.0) * chis + 113.0 / 12.0 * delta * chia
        assert abs(wf.spin_orbit_beta(m1, m2, c1, c2) - alt) < 1e-12


def test_isco_and_band():
    assert abs(wf.f_isco(1.4, 1.4) - 1570.0) < 5.0
    k_lo, k_hi = wf.band(2048.0, 524288, 20.0)
    assert (k_lo, k_hi) == (5120, 262143)
    k_lo, k_hi = wf.band(2048.0, 524288, 20.0, 10.0, 10.0)
    assert k_hi == math.floor(wf.f_isco(10.0, 10.0) / (2048.0 / 524288))


def test_template_support_and_amplitude():
    h = wf.template(1024.0, 16384, 30.0, (1.4, 1.4, 0, 0, 0))
    k = np.nonzero(h)[0]
    assert k[0] == 480 and k[-1] == 8191
    f = k * (1024.0 / 16384)
    assert np.max(np.abs(np.abs(h[k]) - f ** (-7.0 / 6.0))) < 1e-15


def test_tidal_term_lowers_phase_at_high_frequency():
    f = np.array([100.0, 400.0])
    p0 = wf.phase(f, 1.4, 1.3, 0, 0, 0.0, wf.PN_TIDAL)
    p1 = wf.phase(f, 1.4, 1.3, 0, 0, 800.0, wf.PN_TIDAL)
    M = 2.7 * wf.T_SUN
    eta = 1.4 * 1.3 / 2.7 ** 2
    v = (math.pi * M * f) ** (1.0 / 3.0)
    # the tidal term alone is -(3/(128 eta)) (39/2) Lambda v^5
    assert np.allclose(p1 - p0, -3.0 / (128.0 * eta) * 19.5 * 800.0 * v ** 5, rtol=1e-9, atol=1e-12)

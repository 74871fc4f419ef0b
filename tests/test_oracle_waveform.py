"""Pins for the oracle's TaylorF2 phase, using results derived independently of its code:

* (1/2pi) dPsi/df = t_c - tau(f), where tau is the post-Newtonian time to coalescence
  tau = 5 M / (256 eta v^8) [1 + (743/252 + 11 eta/3) v^2 - (32/5)(pi - beta/4) v^3]
  (Peters' chirp time at leading order, with the standard 1PN / 1.5PN corrections);
* the spin-orbit coefficient in its (chi_s, chi_a, delta) form,
  beta = (113/12 - 19 eta/3) chi_s + (113/12) delta chi_a;
* f_ISCO of a 1.4 + 1.4 Msun binary is about 1570 Hz;
* the tidal term: the time shift it puts into (1/2pi) dPsi/df equals the one that energy
  balance gives from the adiabatic-tide binding energy and GW flux of Flanagan & Hinderer
  (Phys. Rev. D 77, 021502(R), 2008), with Lambda~ as defined there (and in Favata, Phys.
  Rev. Lett. 112, 101101, 2014).  The energy and flux below are the physics inputs; the
  phase's -(39/2) Lambda~ v^10 is never used to build the expected value.
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


def tidal_energy_flux(x, m1, m2, lbar1, lbar2):
    """Binding energy E(x) / (eta M), its derivative dE/dx, and GW flux F(x) / eta^2 of a
    circular binary with adiabatic quadrupole tides (Newtonian tidal order; lbar_i =
    lambda_i / M^5 is body i's tidal deformability in units of the total mass),
    x = (M omega)^(2/3):
        E = -(x/2) [1 - 9 (m2/m1 lbar1 + m1/m2 lbar2) x^5]
        F = (32/5) x^5 [1 + 6 ((m1 + 3 m2)/m1 lbar1 + (3 m1 + m2)/m2 lbar2) x^5]
    (the tidal potential -(3/2) lambda_2 m1^2 / r^6 shifts the orbit and the energy; the
    induced quadrupole 3 lambda_2 m1 / r^3 adds to the orbital one mu r^2 in the flux)."""
    ce = 9.0 * (m2 / m1 * lbar1 + m1 / m2 * lbar2)
    e = -0.5 * x * (1.0 - ce * x ** 5)
    de = -0.5 * (1.0 - 6.0 * ce * x ** 5)
    f = 32.0 / 5.0 * x ** 5 * (1.0 + 6.0 * ((m1 + 3 * m2) / m1 * lbar1 + (3 * m1 + m2) / m2 * lbar2) * x ** 5)
    return e, de, f


def lambda_tilde(m1, m2, lbar1, lbar2):
    """Lambda~ = (16/13) [(m1 + 12 m2) m1^4 Lambda1 + (m2 + 12 m1) m2^4 Lambda2] / M^5 with
    Lambda_i = lambda_i / m_i^5, written through lbar_i = lambda_i / M^5."""
    return 16.0 / 13.0 * ((1.0 + 12.0 * m2 / m1) * lbar1 + (1.0 + 12.0 * m1 / m2) * lbar2)


@pytest.mark.parametrize("m1,m2,share1", [(1.4, 1.4, 0.5), (1.6, 1.2, 0.0), (1.9, 1.1, 1.0), (2.4, 1.0, 0.3)])
def test_tidal_phase_term_from_energy_balance(m1, m2, share1):
    """dt/dx = -(dE/dx) / F (energy balance).  The part of t linear in the deformabilities,
    integrated between two frequencies, must equal the change that the tidal term of Psi
    makes in (1/2pi) dPsi/df between the same frequencies."""
    from scipy.integrate import quad
    Mt = (m1 + m2) * wf.T_SUN
    eta = m1 * m2 / (m1 + m2) ** 2
    lam = 700.0
    # split Lambda~ between the bodies: lbar scaled so that lambda_tilde(...) == lam
    unit = lambda_tilde(m1, m2, share1, 1.0 - share1)
    lb1, lb2 = lam * share1 / unit, lam * (1.0 - share1) / unit
    assert abs(lambda_tilde(m1, m2, lb1, lb2) - lam) < 1e-9 * lam

    def dtdx_linear(x):
        # the part of -(dE/dx)/F linear in the deformabilities: a central difference in a
        # scale eps of both (the quadratic part cancels, the cubic one is ~1e-8 relative)
        def g(eps):
            _, de, fl = tidal_energy_flux(x, m1, m2, eps * lb1, eps * lb2)
            return -de / fl
        d = 1e-2
        return (g(d) - g(-d)) / (2.0 * d) * Mt / eta      # t in seconds: E ~ eta M, F ~ eta^2

    def t_tidal_from_phase(f):
        # (1/2pi) d/df of the phase difference made by the tidal term (fourth-order difference)
        h = 1e-4 * f
        dph = lambda ff: (wf.phase(ff, m1, m2, 0, 0, lam, wf.PN_TIDAL) - wf.phase(ff, m1, m2, 0, 0, 0.0, wf.PN_TIDAL))
        return (-dph(f + 2 * h) + 8 * dph(f + h) - 8 * dph(f - h) + dph(f - 2 * h)) / (12 * h) / (2 * math.pi)

    x_of = lambda f: (math.pi * Mt * f) ** (2.0 / 3.0)
    for f1, f2 in ((40.0, 200.0), (100.0, 500.0), (300.0, 900.0)):
        expect = quad(dtdx_linear, x_of(f1), x_of(f2), epsabs=0, epsrel=1e-10)[0]
        got = t_tidal_from_phase(f2) - t_tidal_from_phase(f1)
        assert abs(got - expect) <= 1e-5 * abs(expect), (f1, f2, got, expect)
        assert expect < 0          # tides shorten the remaining time: the shift grows with f

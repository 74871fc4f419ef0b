"""TaylorF2 templates in FP64 (oracle; test infrastructure).

The matched filter of Eq. 1 correlates the data with a frequency-domain template h(f).
The workloads use the stationary-phase TaylorF2 chirp:

  h(f)   = f^(-7/6) exp(-i Psi(f))   for f_low <= f <= f_ISCO, zero elsewhere
  Psi(f) = 2 pi f t_c - phi_c - pi/4
           + 3/(128 eta v^5) [1 + (3715/756 + 55 eta/9) v^2 + (4 beta - 16 pi) v^3
                              - (39/2) Lambda v^10]
  v = (pi M f)^(1/3),  M = (m1 + m2) G Msun / c^3,  eta = m1 m2 / (m1 + m2)^2
  beta = (1/12) sum_i [113 (m_i/M)^2 + 75 eta] chi_i      (aligned-spin 1.5PN spin-orbit)
  f_ISCO = 1 / (6^(3/2) pi M)

with t_c = phi_c = 0.  The amplitude carries no mass prefactor: every SNR is normalised by
the template's own sigma, so the overall amplitude cancels and the ratio of two templates
has unit modulus wherever both are non-zero (the ratio of Eq. 2).
"""
import math

import numpy as np

T_SUN = 4.925490947641267e-6
PN_SO = 1
PN_TIDAL = 2


def total_mass_s(m1, m2):
    return (m1 + m2) * T_SUN


def f_isco(m1, m2):
    return 1.0 / (6.0 ** 1.5 * math.pi * total_mass_s(m1, m2))


def spin_orbit_beta(m1, m2, chi1, chi2):
    mtot = m1 + m2
    eta = m1 * m2 / mtot ** 2
    return ((113.0 * (m1 / mtot) ** 2 + 75.0 * eta) * chi1
            + (113.0 * (m2 / mtot) ** 2 + 75.0 * eta) * chi2) / 12.0


def phase(f, m1, m2, chi1=0.0, chi2=0.0, lam=0.0, pn_flags=0, tc=0.0, phic=0.0):
    """Psi(f) of the TaylorF2 template, FP64."""
    f = np.asarray(f, dtype=np.float64)
    mt = total_mass_s(m1, m2)
    eta = m1 * m2 / (m1 + m2) ** 2
    v = (math.pi * mt * f) ** (1.0 / 3.0)
    beta = spin_orbit_beta(m1, m2, chi1, chi2) if (pn_flags & PN_SO) else 0.0
    lam_eff = lam if (pn_flags & PN_TIDAL) else 0.0
    bracket = (1.0
               + (3715.0 / 756.0 + 55.0 * eta / 9.0) * v ** 2
               + (4.0 * beta - 16.0 * math.pi) * v ** 3
               - (39.0 / 2.0) * lam_eff * v ** 10)
    return 2.0 * math.pi * f * tc - phic - math.pi / 4.0 + 3.0 / (128.0 * eta * v ** 5) * bracket


def band(fs, n, f_low, m1=None, m2=None):
    """Inclusive bin range [k_lo, k_hi] of a template (or of the data when no masses are
    given): k_lo = ceil(f_low/df), k_hi = min(n/2 - 1, floor(f_ISCO/df)).  DC and Nyquist
    are always excluded."""
    df = fs / n
    k_lo = int(math.ceil(f_low / df - 1e-12))
    k_hi = n // 2 - 1
    if m1 is not None:
        k_hi = min(k_hi, int(math.floor(f_isco(m1, m2) / df)))
    return k_lo, k_hi


def template(fs, n, f_low, params, pn_flags=0) -> np.ndarray:
    """h(f_k), k = 0..n/2, complex128, zero outside the template's band."""
    m1, m2, chi1, chi2, lam = [float(x) for x in params]
    k_lo, k_hi = band(fs, n, f_low, m1, m2)
    h = np.zeros(n // 2 + 1, dtype=np.complex128)
    if k_hi < k_lo:
        return h
    f = np.arange(k_lo, k_hi + 1, dtype=np.float64) * (fs / n)
    psi = phase(f, m1, m2, chi1, chi2, lam, pn_flags)
    h[k_lo:k_hi + 1] = f ** (-7.0 / 6.0) * np.exp(-1j * psi)
    return h

"""Seeded generators: PSD samples, template bank, references, coloured noise, injections.

Conventions (shared with every consumer of these arrays):
  * frequency grid f_k = k * df, df = fs / n, k = 0 .. n/2 (one-sided spectrum);
  * the data spectrum is zero outside the data band k in [ceil(f_low/df), n/2 - 1]
    (DC and Nyquist excluded);
  * noise bins are sqrt(S_k / (4 df)) * (a_k + i b_k) with a_k, b_k standard normal,
    drawn from numpy's PCG64 in k order, a before b;
  * an injection of optimal SNR rho at sample m0 with phase phi adds
    A * h(f_k) * exp(-2 pi i k m0 / n) * exp(i phi) with A = rho / sigma(h),
    sigma^2 = 4 df sum_k |h_k|^2 / S_k over the injected waveform's band.
"""
from dataclasses import dataclass
import math
from typing import List, Tuple

import numpy as np

from .configs import Config, PN_SO, PN_TIDAL

T_SUN = 4.925490947641267e-6  # G M_sun / c^3 in seconds


def psd_analytic(f):
    """Analytic one-sided PSD S(x) = x^-4.14 - 5 x^-2 + 111 (1 - x^2 + x^4/2) / (1 + x^2/2),
    x = f / 215 Hz, used unscaled (the SNR does not depend on the PSD's overall scale)."""
    x = np.asarray(f, dtype=np.float64) / 215.0
    return x ** -4.14 - 5.0 / x ** 2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2)


def chirp_mass(m1, m2):
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2


def band_low_index(fs: float, n: int, f_low: float) -> int:
    return int(math.ceil(f_low / (fs / n) - 1e-12))


@dataclass
class Bank:
    """Template-bank parameters (float64) and the template -> reference association."""
    m1: np.ndarray
    m2: np.ndarray
    chi1: np.ndarray
    chi2: np.ndarray
    lam: np.ndarray
    ref_m1: np.ndarray
    ref_m2: np.ndarray
    ref_chi1: np.ndarray
    ref_chi2: np.ndarray
    ref_lam: np.ndarray
    ref_of_tmpl: np.ndarray   # int32 [n_tmpl]
    ref_tmpl_index: np.ndarray  # int32 [n_ref]: the bank slot each reference copies (-1: none)

    @property
    def n_tmpl(self):
        return len(self.m1)

    @property
    def n_ref(self):
        return len(self.ref_m1)

    def params(self) -> np.ndarray:
        """Template parameters as float64 [n_tmpl, 5] = (m1, m2, chi1, chi2, lambda_tilde)."""
        return np.stack([self.m1, self.m2, self.chi1, self.chi2, self.lam], axis=1).copy()

    def ref_params(self) -> np.ndarray:
        return np.stack([self.ref_m1, self.ref_m2, self.ref_chi1, self.ref_chi2, self.ref_lam],
                        axis=1).copy()

    def subset(self, idx) -> "Bank":
        idx = np.asarray(idx)
        return Bank(self.m1[idx], self.m2[idx], self.chi1[idx], self.chi2[idx], self.lam[idx],
                    self.ref_m1, self.ref_m2, self.ref_chi1, self.ref_chi2, self.ref_lam,
                    self.ref_of_tmpl[idx].astype(np.int32), self.ref_tmpl_index)


@dataclass
class Data:
    dtilde: np.ndarray        # complex128 [n/2+1]
    psd: np.ndarray           # float64 [n/2+1]
    injections: List[Tuple[int, float, float, int]]  # (sample m0, snr, phase, bank slot)
    k_lo: int


def make_bank(cfg: Config, n_tmpl: int = None) -> Bank:
    n = cfg.n_tmpl if n_tmpl is None else n_tmpl
    rng = np.random.default_rng(cfg.seeds[0])
    m = rng.uniform(cfg.m_range[0], cfg.m_range[1], size=(n, 2))
    m1 = np.maximum(m[:, 0], m[:, 1])
    m2 = np.minimum(m[:, 0], m[:, 1])
    if cfg.chi_range is not None:
        chi = rng.uniform(cfg.chi_range[0], cfg.chi_range[1], size=(n, 2))
        chi1, chi2 = chi[:, 0].copy(), chi[:, 1].copy()
    else:
        chi1 = np.zeros(n)
        chi2 = np.zeros(n)
    if cfg.lambda_range is not None:
        lam = rng.uniform(cfg.lambda_range[0], cfg.lambda_range[1], size=n)
    else:
        lam = np.zeros(n)

    if cfg.c1_slots:
        # one reference at the centre of the mass range; slot 0 is the reference itself,
        # slot 1 the reference with m1 + 0.001 Msun (a template the short filter can match)
        mc = 0.5 * (cfg.m_range[0] + cfg.m_range[1])
        m1[0], m2[0] = mc, mc
        m1[1], m2[1] = mc + 0.001, mc
        chi1[:2] = 0.0
        chi2[:2] = 0.0
        lam[:2] = 0.0
        ref_idx = np.array([0], dtype=np.int32)
        ref_of = np.zeros(n, dtype=np.int32)
    else:
        mcs = chirp_mass(m1, m2)
        order = np.argsort(mcs, kind="stable")
        groups = np.array_split(order, min(cfg.n_ref, n))
        ref_idx = np.array([g[len(g) // 2] for g in groups], dtype=np.int32)
        ref_mc = mcs[ref_idx]
        # nearest reference in chirp mass, ties to the lower reference index
        d = np.abs(mcs[:, None] - ref_mc[None, :])
        ref_of = np.argmin(d, axis=1).astype(np.int32)
    return Bank(m1, m2, chi1, chi2, lam,
                m1[ref_idx].copy(), m2[ref_idx].copy(), chi1[ref_idx].copy(),
                chi2[ref_idx].copy(), lam[ref_idx].copy(), ref_of, ref_idx)


def make_training_bank(cfg: Config, bank: Bank, n_train: int) -> Bank:
    """Templates from cfg's parameter distribution with the training seed 5000 + c, assigned to
    `bank`'s references by nearest chirp mass (the learned-tap networks' training set)."""
    rng = np.random.default_rng(5000 + cfg.index)
    m = rng.uniform(cfg.m_range[0], cfg.m_range[1], size=(n_train, 2))
    m1 = np.maximum(m[:, 0], m[:, 1])
    m2 = np.minimum(m[:, 0], m[:, 1])
    z = np.zeros(n_train)
    chi1, chi2, lam = z.copy(), z.copy(), z.copy()
    if cfg.chi_range is not None:
        chi = rng.uniform(cfg.chi_range[0], cfg.chi_range[1], size=(n_train, 2))
        chi1, chi2 = chi[:, 0].copy(), chi[:, 1].copy()
    if cfg.lambda_range is not None:
        lam = rng.uniform(cfg.lambda_range[0], cfg.lambda_range[1], size=n_train)
    ref_mc = chirp_mass(bank.ref_m1, bank.ref_m2)
    d = np.abs(chirp_mass(m1, m2)[:, None] - ref_mc[None, :])
    ref_of = np.argmin(d, axis=1).astype(np.int32)
    return Bank(m1, m2, chi1, chi2, lam, bank.ref_m1, bank.ref_m2, bank.ref_chi1, bank.ref_chi2, bank.ref_lam,
                ref_of, bank.ref_tmpl_index)


def dense_bank(ref_params, n_per_ref: int, delta_mc: float, seed: int, q_range=(0.8, 1.0),
               chi_range=(-0.05, 0.05), lam_range=(0.0, 2000.0)) -> Bank:
    """The dense-reference regime of the paper (references about 1 % of the bank, each
    template close to its reference): for each reference, n_per_ref templates with chirp mass
    uniform within a relative +-delta_mc of the reference's, mass ratio q = m2/m1 uniform in
    q_range, spins and Lambda~ uniform.  Templates are grouped by reference."""
    ref = np.asarray(ref_params, dtype=np.float64).reshape(-1, 5)
    rng = np.random.default_rng(seed)
    out, ref_of = [], []
    for r, p in enumerate(ref):
        mc0 = float(chirp_mass(p[0], p[1]))
        mc = mc0 * (1.0 + delta_mc * rng.uniform(-1.0, 1.0, n_per_ref))
        q = rng.uniform(q_range[0], q_range[1], n_per_ref)
        m1 = mc * (1.0 + q) ** 0.2 / q ** 0.6
        m2 = q * m1
        c = rng.uniform(chi_range[0], chi_range[1], (n_per_ref, 2))
        lam = rng.uniform(lam_range[0], lam_range[1], n_per_ref)
        out.append(np.stack([m1, m2, c[:, 0], c[:, 1], lam], axis=1))
        ref_of.append(np.full(n_per_ref, r, dtype=np.int32))
    P = np.concatenate(out)
    return Bank(P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy(), P[:, 3].copy(), P[:, 4].copy(),
                ref[:, 0].copy(), ref[:, 1].copy(), ref[:, 2].copy(), ref[:, 3].copy(), ref[:, 4].copy(),
                np.concatenate(ref_of), np.full(len(ref), -1, dtype=np.int32))


def _inject(f, m1, m2, chi1, chi2, lam, pn_flags, f_low):
    """Frequency-domain TaylorF2 chirp for the injected signal (data synthesis only):
    amplitude f^(-7/6) between f_low and the Schwarzschild ISCO, stationary-phase phase
    through 1.5PN (plus spin-orbit and 5PN tidal terms when enabled), t_c = phi_c = 0."""
    mt = (m1 + m2) * T_SUN
    eta = m1 * m2 / (m1 + m2) ** 2
    out = np.zeros(len(f), dtype=np.complex128)
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * mt)
    sel = (f >= f_low) & (f <= f_isco)
    fs_ = f[sel]
    v = np.cbrt(math.pi * mt * fs_)
    beta = 0.0
    if pn_flags & PN_SO:
        q1, q2 = m1 / (m1 + m2), m2 / (m1 + m2)
        beta = ((113.0 * q1 * q1 + 75.0 * eta) * chi1 + (113.0 * q2 * q2 + 75.0 * eta) * chi2) / 12.0
    series = (1.0 + (3715.0 / 756.0 + 55.0 * eta / 9.0) * v ** 2
              + (4.0 * beta - 16.0 * math.pi) * v ** 3)
    if pn_flags & PN_TIDAL:
        series = series - 19.5 * lam * v ** 10
    psi = -math.pi / 4.0 + 3.0 / (128.0 * eta) * series / v ** 5
    out[sel] = fs_ ** (-7.0 / 6.0) * np.exp(-1j * psi)
    return out


def make_data(cfg: Config, bank: Bank, n: int = None, inject: bool = True,
              noise: bool = True) -> Data:
    n = cfg.n if n is None else n
    df = cfg.fs / n
    nf = n // 2 + 1
    f = np.arange(nf, dtype=np.float64) * df
    psd = np.empty(nf)
    psd[1:] = psd_analytic(f[1:])
    psd[0] = psd[1]
    k_lo = band_low_index(cfg.fs, n, cfg.f_low)
    k_hi = n // 2 - 1
    d = np.zeros(nf, dtype=np.complex128)
    if noise:
        rng = np.random.default_rng(cfg.seeds[1])
        ab = rng.standard_normal(size=(k_hi - k_lo + 1, 2))
        amp = np.sqrt(psd[k_lo:k_hi + 1] / (4.0 * df))
        d[k_lo:k_hi + 1] = amp * (ab[:, 0] + 1j * ab[:, 1])
    injections = []
    if inject and cfg.n_inj > 0:
        rng = np.random.default_rng(cfg.seeds[2])
        dur = n / cfg.fs
        for i in range(cfg.n_inj):
            if cfg.c1_slots:
                slot, snr, phase, t0 = 1, cfg.inj_snr[0], 0.0, 10.0
            else:
                slot = int(rng.integers(bank.n_tmpl))
                snr = float(rng.uniform(cfg.inj_snr[0], cfg.inj_snr[1]))
                phase = float(rng.uniform(0.0, 2.0 * math.pi))
                t0 = (20.0 + 30.0 * i) % dur
            m0 = int(round(t0 * cfg.fs)) % n
            h = _inject(f, bank.m1[slot], bank.m2[slot], bank.chi1[slot], bank.chi2[slot],
                        bank.lam[slot], cfg.pn_flags, cfg.f_low)
            h[:k_lo] = 0.0
            h[k_hi + 1:] = 0.0
            sig = math.sqrt(4.0 * df * np.sum(np.abs(h[1:]) ** 2 / psd[1:]))
            k = np.arange(nf)
            d += (snr / sig) * h * np.exp(-2j * math.pi * k * m0 / n) * np.exp(1j * phase)
            injections.append((m0, snr, phase, slot))
    return Data(d, psd, injections, k_lo)


def make_workload(cfg: Config, n_tmpl: int = None, n: int = None, **kw):
    bank = make_bank(cfg, n_tmpl)
    data = make_data(cfg, bank, n=n, **kw)
    return bank, data

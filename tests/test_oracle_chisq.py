"""Pins for the sub-band chi^2 through the ratio filter (oracle/chisq.py, Sec. VI).

* linearity: the sub-band SNRs add up to the template's SNR of Eq. 3 (ratio.snr_series);
* the edges split the reference's SNR into p equal shares (to one bin's weight) and the
  effective template's band shares u_b add to 1;
* a noise-free signal equal to the effective template gives z_b = u_b z at its time, i.e.
  chi^2 = 0 there;
* pure Gaussian noise gives mean chi^2 = 2 (p - 1) (its degrees of freedom);
* a loud signal of a different chirp (a glitch-like mismatch) gives chi^2 far above 2 (p - 1).
"""
import math

import numpy as np
import pytest

import workload
from oracle import chisq, matched, ratio, waveform as wf

P = 8


@pytest.fixture(scope="module")
def grid():
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg, noise=True)
    return cfg, bank, data


def _setup(cfg, bank, data, j, dtilde, K=64):
    df = cfg.fs / cfg.n
    ref = bank.ref_params()[0]
    h_ref = wf.template(cfg.fs, cfg.n, cfg.f_low, ref)
    o = ratio.design(cfg.fs, cfg.n, cfg.f_low, bank.params()[j], ref, data.psd, K, with_match=False)
    edges = chisq.band_edges(h_ref, data.psd, df, P)
    qb = chisq.band_series(dtilde, h_ref, data.psd, df, cfg.n, edges)
    Cb = chisq.band_autocorr(h_ref, data.psd, df, cfg.n, edges, K - 1)
    return h_ref, o, edges, qb, Cb


def test_linearity_and_shares(grid):
    cfg, bank, data = grid
    df = cfg.fs / cfg.n
    j = 5
    h_ref, o, edges, qb, Cb = _setup(cfg, bank, data, j, data.dtilde)
    t = np.arange(0, cfg.n, 97)
    chi2, zb, u = chisq.subband_chi2(qb, o["taps"], o["lag"], o["sigma_eff"], Cb, t)
    q_ref = matched.filter_unnormalised(data.dtilde, h_ref, data.psd, df, cfg.n)
    z = ratio.snr_series(q_ref, o["taps"], o["lag"], o["sigma_eff"])[t]
    assert np.max(np.abs(zb.sum(axis=0) - z)) <= 1e-11 * np.max(np.abs(z))
    assert abs(u.sum() - 1) < 1e-12
    w = chisq.band_weights(h_ref, data.psd, df)
    W = w.sum()
    for b in range(P):
        share = w[edges[b]:edges[b + 1]].sum()
        assert abs(share - W / P) <= w.max() + 1e-12 * W
    assert np.all(np.diff(edges) > 0)


def test_effective_template_signal_has_zero_chi2(grid):
    cfg, bank, data = grid
    df = cfg.fs / cfg.n
    j = 7
    ref = bank.ref_params()[0]
    h_ref = wf.template(cfg.fs, cfg.n, cfg.f_low, ref)
    o = ratio.design(cfg.fs, cfg.n, cfg.f_low, bank.params()[j], ref, data.psd, 64, with_match=False)
    A = ratio.effective_response(o["taps"], o["lag"], cfg.n)[: cfg.n // 2 + 1]
    h_eff = h_ref * np.conj(A)
    m0 = 3000
    k = np.arange(cfg.n // 2 + 1)
    d = 20.0 * h_eff * np.exp(-2j * math.pi * k * m0 / cfg.n) / o["sigma_eff"]
    _, _, edges, qb, Cb = _setup(cfg, bank, data, j, d)
    chi2, zb, u = chisq.subband_chi2(qb, o["taps"], o["lag"], o["sigma_eff"], Cb, [m0])
    z = zb.sum(axis=0)
    assert abs(abs(z[0]) - 20.0) < 1e-9
    assert chi2[0] < 1e-18 * abs(z[0]) ** 2        # at the signal's time: z_b = u_b z exactly


def test_noise_mean_is_degrees_of_freedom():
    cfg = workload.small_config(2, n=65536, n_inj=0)
    bank, data = workload.make_workload(cfg, n_tmpl=8)
    h_ref, o, edges, qb, Cb = _setup(cfg, bank, data, 3, data.dtilde)
    t = np.arange(0, cfg.n, 8)
    chi2, _, _ = chisq.subband_chi2(qb, o["taps"], o["lag"], o["sigma_eff"], Cb, t)
    assert abs(np.mean(chi2) / (2 * (P - 1)) - 1) < 0.06


def test_mismatched_loud_signal_has_large_chi2(grid):
    cfg, bank, data = grid
    df = cfg.fs / cfg.n
    j = 7
    other = (1.2, 1.2, 0.0, 0.0, 0.0)        # a different chirp, injected loud
    h_o = wf.template(cfg.fs, cfg.n, cfg.f_low, other)
    m0 = 5000
    k = np.arange(cfg.n // 2 + 1)
    sig = math.sqrt(matched.sigma_sq(h_o, data.psd, df))
    d = data.dtilde + 200.0 / sig * h_o * np.exp(-2j * math.pi * k * m0 / cfg.n)
    h_ref, o, edges, qb, Cb = _setup(cfg, bank, data, j, d)
    q_ref = matched.filter_unnormalised(d, h_ref, data.psd, df, cfg.n)
    z = ratio.snr_series(q_ref, o["taps"], o["lag"], o["sigma_eff"])
    t_pk = int(np.argmax(np.abs(z)))
    chi2, _, _ = chisq.subband_chi2(qb, o["taps"], o["lag"], o["sigma_eff"], Cb, [t_pk])
    assert abs(z[t_pk]) > 8
    assert chi2[0] > 10 * 2 * (P - 1)

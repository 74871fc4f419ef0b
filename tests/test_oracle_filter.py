"""Pins for the oracle's matched filter and ratio-filter path.

* noise-free injection: |z| peaks at the injected sample with z = rho_inj exp(i phi0);
* pure noise: mean |z|^2 = 2 within 4 exact standard errors (complex SNR, chi^2 with 2 dof);
* Eq. 3 associativity: with K = N unwindowed taps the ratio path equals FINDCHIRP;
* identity template: G == 1, taps = delta at K/2, lag -K/2, z_ratio = z_ref;
* Eqs. 5-6: the Parseval quadratic form equals the frequency-domain sum, and tends to
  sigma(h_j) as K -> N;
* Tukey window equals scipy's; trigger reduction equals a brute-force loop.
"""
import math

import numpy as np
import pytest

import workload
from oracle import matched, ratio, triggers, waveform as wf

FS, N, FLOW = 256.0, 4096, 20.0
DF = FS / N


def psd_grid(n=N, fs=FS):
    f = np.arange(n // 2 + 1) * (fs / n)
    S = np.empty(n // 2 + 1)
    S[1:] = workload.psd_analytic(f[1:])
    S[0] = S[1]
    return S


def test_injection_closed_form():
    S = psd_grid()
    p = (1.4, 1.3, 0, 0, 0)
    h = wf.template(FS, N, FLOW, p)
    m0, rho, phi0 = 1234, 11.0, 0.7
    k = np.arange(N // 2 + 1)
    sig = math.sqrt(matched.sigma_sq(h, S, DF))
    d = rho / sig * h * np.exp(-2j * math.pi * k * m0 / N) * np.exp(1j * phi0)
    z = matched.findchirp(d, h, S, DF, N)
    assert int(np.argmax(np.abs(z))) == m0
    assert abs(z[m0] - rho * np.exp(1j * phi0)) < 1e-10


def test_workload_injection_recovered_by_oracle_template():
    cfg = workload.small_config(1, n_inj=1)
    bank, data = workload.make_workload(cfg, noise=False)
    m0, snr, phi, slot = data.injections[0]
    h = wf.template(cfg.fs, cfg.n, cfg.f_low, bank.params()[slot])
    z = matched.findchirp(data.dtilde, h, data.psd, cfg.fs / cfg.n, cfg.n)
    assert int(np.argmax(np.abs(z))) == m0
    assert abs(z[m0] - snr * np.exp(1j * phi)) < 1e-9 * snr


def test_noise_mean_snr_squared_is_two():
    cfg = workload.small_config(2, n=65536, n_inj=0)
    bank, data = workload.make_workload(cfg, n_tmpl=4)
    df = cfg.fs / cfg.n
    h = wf.template(cfg.fs, cfg.n, cfg.f_low, bank.params()[0])
    z = matched.findchirp(data.dtilde, h, data.psd, df, cfg.n)
    mean = np.mean(np.abs(z) ** 2)
    nz = np.nonzero(h)[0]
    sig2 = matched.sigma_sq(h, data.psd, df)
    se = 2.0 * 4.0 * df * math.sqrt(np.sum(np.abs(h[nz]) ** 4 / data.psd[nz] ** 2)) / sig2
    assert abs(mean - 2.0) < 4.0 * se, (mean, se)
    # tail: P(|z|^2 > 25) = exp(-12.5) for chi^2_2
    assert np.mean(np.abs(z) ** 2 > 25.0) < 1e-3


def _tmpl_ref_pair():
    return (1.43, 1.38, 0, 0, 0), (1.4, 1.4, 0, 0, 0)


def test_ratio_path_with_full_length_taps_equals_findchirp(rng):
    """Eq. 3: F^-1[conj(h/h_ref)] convolved with (s|h_ref) is (s|h) exactly when nothing is cut."""
    n = 1024
    S = psd_grid(n)
    tp, rp = _tmpl_ref_pair()
    d = np.zeros(n // 2 + 1, complex)
    k_lo, k_hi = wf.band(FS, n, FLOW)
    d[k_lo:k_hi + 1] = rng.standard_normal(k_hi - k_lo + 1) + 1j * rng.standard_normal(k_hi - k_lo + 1)
    df = FS / n
    h_j = wf.template(FS, n, FLOW, tp)
    h_r = wf.template(FS, n, FLOW, rp)
    q_j = matched.filter_unnormalised(d, h_j, S, df, n)
    q_r = matched.filter_unnormalised(d, h_r, S, df, n)
    g = ratio.impulse_response(ratio.ratio_spectrum(FS, n, FLOW, tp, rp))
    s = ratio.choose_lag(ratio.window_energy(g, np.ones(n)), n)
    rho = g[(s + np.arange(n)) % n]
    qhat = ratio.ratio_fir(q_r, rho, s)
    assert np.max(np.abs(qhat - q_j)) < 1e-11 * np.max(np.abs(q_j))
    # and its sigma_eff is sigma(h_j), its match 1
    C = ratio.autocorrelation(h_r, S, df, n, n - 1)
    assert abs(ratio.sigma_eff_sq_parseval(rho, C) / matched.sigma_sq(h_j, S, df) - 1) < 1e-11
    assert abs(ratio.tap_match(h_j, rho, s, h_r, S, df, n) - 1.0) < 1e-12


def test_identity_template_gives_delta_taps(rng):
    n, K = 4096, 64
    S = psd_grid(n)
    rp = (1.4, 1.4, 0, 0, 0)
    G = ratio.ratio_spectrum(FS, n, FLOW, rp, rp)
    assert np.max(np.abs(G - 1.0)) == 0.0
    out = ratio.design(FS, n, FLOW, rp, rp, S, K, 0.1)
    assert out["lag"] == -K // 2
    delta = np.zeros(K)
    delta[K // 2] = 1.0
    assert np.max(np.abs(out["taps"] - delta)) < 1e-14
    h_r = wf.template(FS, n, FLOW, rp)
    assert abs(out["sigma_eff"] ** 2 / matched.sigma_sq(h_r, S, FS / n) - 1) < 1e-12
    assert abs(out["match"] - 1) < 1e-12
    d = np.zeros(n // 2 + 1, complex)
    k_lo, k_hi = wf.band(FS, n, FLOW)
    d[k_lo:k_hi + 1] = rng.standard_normal(k_hi - k_lo + 1) + 1j * rng.standard_normal(k_hi - k_lo + 1)
    q_r = matched.filter_unnormalised(d, h_r, S, FS / n, n)
    z_ratio = ratio.snr_series(q_r, out["taps"], out["lag"], out["sigma_eff"])
    z_ref = matched.findchirp(d, h_r, S, FS / n, n)
    assert np.max(np.abs(z_ratio - z_ref)) < 1e-14 * np.max(np.abs(z_ref)) * 10


@pytest.mark.parametrize("K", [32, 128])
def test_sigma_eff_parseval_equals_frequency_sum(K):
    n = 4096
    S = psd_grid(n)
    tp, rp = _tmpl_ref_pair()
    out = ratio.design(FS, n, FLOW, tp, rp, S, K, 0.1, with_match=False)
    h_r = wf.template(FS, n, FLOW, rp)
    freq = ratio.sigma_eff_sq_freq(out["taps"], out["lag"], h_r, S, FS / n, n)
    assert abs(out["sigma_eff"] ** 2 / freq - 1) < 1e-12


def test_tukey_matches_scipy():
    sw = pytest.importorskip("scipy.signal.windows")
    for K in (1, 2, 7, 32, 64, 251, 512):
        for a in (0.0, 0.1, 0.5, 1.0):
            assert np.max(np.abs(ratio.tukey(K, a) - sw.tukey(K, a, sym=True))) < 1e-14


def test_ratio_fir_at_matches_full_series(rng):
    q = rng.standard_normal(512) + 1j * rng.standard_normal(512)
    rho = rng.standard_normal(16) + 1j * rng.standard_normal(16)
    full = ratio.ratio_fir(q, rho, -7)
    t = np.array([0, 1, 100, 511])
    assert np.max(np.abs(ratio.ratio_fir_at(q, rho, -7, t) - full[t])) < 1e-13


def test_ratio_fir_is_brute_force_convolution(rng):
    n, K, s = 64, 5, -3
    q = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    rho = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    out = ratio.ratio_fir(q, rho, s)
    for m in range(n):
        acc = 0j
        for k in range(K):
            acc += rho[k] * q[(m - s - k) % n]
        assert abs(out[m] - acc) < 1e-13


def test_trigger_reduction_matches_bruteforce(rng):
    for trial in range(20):
        n = int(rng.integers(50, 400))
        W = int(rng.integers(1, 40))
        z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 3
        z = np.round(z, 1)                     # rounding creates exact ties
        a = triggers.window_triggers(z, W, 9.0)
        b = triggers.window_triggers_bruteforce(z, W, 9.0)
        assert [(x["w"], x["t"]) for x in a] == [(x["w"], x["t"]) for x in b]
        assert all(abs(x["p"] - y["p"]) < 1e-12 for x, y in zip(a, b))


def test_energy_span_and_bucket():
    g = np.zeros(256, complex)
    g[250:256] = 1.0
    g[0:4] = 1.0
    assert ratio.energy_span(g, 1.0) == 10
    assert ratio.k_bucket(g, (4, 8, 16, 32), 1.0) == 16


@pytest.mark.parametrize("K,n,s", [(64, 16384, -37), (512, 16384, 211), (3, 4096, 0), (200, 1024, -5)])
def test_overlap_save_blocks_reproduce_the_circular_fir(rng, K, n, s):
    """Reading of the block-FFT realisation (Table II's form): with off = (s + K - 1) mod n,
    c[m] = rho[K-1-m], blocks of L = M - K + 1 outputs (M = 2048) starting at u0 = b L and
    x_b[i] = q[(u0 + i) mod n], the unnormalised inverse DFT of X_b P (P = IDFT_M(c) / M)
    gives qhat[(u0 + l + off) mod n] for l < L: every output of the direct circular FIR of
    Eq. 3, exactly once, including blocks that run past the end of the segment (and M > n)."""
    M = 2048
    q = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    rho = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    direct = ratio.ratio_fir(q, rho, s)
    off = (s + K - 1) % n
    c = np.zeros(M, dtype=np.complex128)
    c[:K] = rho[::-1]
    P = np.fft.ifft(c)                       # (1/M) sum_m c[m] e^{+2 pi i k m / M}
    L = M - K + 1
    got = np.full(n, np.nan + 0j)
    for b in range(-(-n // L)):
        u0 = b * L
        x = q[(u0 + np.arange(M)) % n]
        y = np.fft.ifft(np.fft.fft(x) * P) * M
        l = np.arange(min(L, n - u0))
        got[(u0 + l + off) % n] = y[l]
    assert not np.isnan(got).any()
    assert np.max(np.abs(got - direct)) <= 1e-11 * np.max(np.abs(direct))


def test_streaming_windows_tile_the_series(rng):
    """Reading of the streaming form (Sec. VII.A): the outputs u of windows [w0, w0 + B), taken
    with their true times (u + off) mod n, cover the direct circular FIR exactly once."""
    n, K, s, B = 8192, 64, 17, 2048
    q = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    rho = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    direct = ratio.ratio_fir(q, rho, s)
    off = (s + K - 1) % n
    seen = np.zeros(n, dtype=int)
    for w0 in range(0, n, B):
        u = np.arange(w0, w0 + B)
        t = (u + off) % n
        seen[t] += 1
        # the window needs q[u .. u + K - 1] only (the K-sample halo)
        win = np.array([np.sum(rho[::-1] * q[(uu + np.arange(K)) % n]) for uu in u[:8]])
        assert np.allclose(win, direct[t[:8]], rtol=1e-12, atol=1e-12)
    assert np.all(seen == 1)


def test_autocorrelation_equals_its_defining_sum(rng):
    """C_r[l] = sum_k 4 df |h_k|^2 / S_k exp(+2 pi i k l / n) (Eq. 6 on the sample grid),
    summed term by term for every lag, against the oracle's inverse-FFT evaluation."""
    from oracle import ratio, waveform as wf
    fs, n, f_low = 1024.0, 4096, 30.0
    df = fs / n
    h = wf.template(fs, n, f_low, (1.4, 1.3, 0, 0, 0))
    f = np.arange(n // 2 + 1) * df
    psd = 1.0 + (f / 200.0) ** 2 + rng.uniform(0.0, 0.1, len(f))
    C = ratio.autocorrelation(h, psd, df, n, 100)
    k = np.nonzero(h)[0]
    wgt = 4.0 * df * np.abs(h[k]) ** 2 / psd[k]
    for i, l in enumerate(range(-100, 101)):
        direct = np.sum(wgt * np.exp(2j * np.pi * k * l / n))
        assert abs(C[i] - direct) <= 1e-12 * np.sum(wgt)

"""Pins for the chi^2-fitted ridge taps (oracle/fit.py, Sec. V.A).

* the normal-equation solution equals a weighted least-squares solve of the explicit
  over-determined system (rows sqrt(w_k) exp(-2 pi i k (s+n)/N), ridge rows sqrt(lam) I);
* the closed-form match equals the FFT-path tap match of ratio.tap_match;
* the identity template (G = 1) is fitted exactly on the band (match 1, chi^2 ~ 0) by the
  minimum-norm taps, whose norm is below the delta's: the band-limited weight leaves a null
  space and the ridge picks its smallest member;
* at the same K and lag the fitted taps match the template at least as well as the windowed
  taps (least squares is optimal), and strictly better on a chirp-mass offset;
* a larger ridge shrinks the taps' norm and never lowers chi^2;
* the dynamic K is the smallest bucket whose fitted match reaches the target.
"""
import math

import numpy as np
import pytest

import workload
from oracle import fit, ratio, waveform as wf

FS, N, FLOW = 256.0, 4096, 20.0
DF = FS / N
REF = (1.4, 1.4, 0.0, 0.0, 0.0)


def psd_grid():
    f = np.arange(N // 2 + 1) * DF
    S = np.empty(N // 2 + 1)
    S[1:] = workload.psd_analytic(f[1:])
    S[0] = S[1]
    return S


@pytest.fixture(scope="module")
def S():
    return psd_grid()


def chi2(rho, G, w, s, lam):
    k = np.arange(len(w))
    A = np.exp(-2j * math.pi * np.outer(k, s + np.arange(len(rho))) / N) @ rho
    return float(np.sum(w * np.abs(G[: len(w)] - A) ** 2) + lam * np.sum(np.abs(rho) ** 2))


def test_normal_equations_equal_weighted_least_squares(S):
    tmpl = (1.42, 1.39, 0.0, 0.0, 0.0)
    K, eps = 48, 1e-5
    out = fit.design(FS, N, FLOW, tmpl, REF, S, K, eps)
    G = ratio.ratio_spectrum(FS, N, FLOW, tmpl, REF)
    h_ref = wf.template(FS, N, FLOW, REF)
    w = fit.weights(h_ref, S, DF)
    nz = np.nonzero(w)[0]
    s = out["lag"]
    rows = np.sqrt(w[nz])[:, None] * np.exp(-2j * math.pi * np.outer(nz, s + np.arange(K)) / N)
    lam = eps * out["C"][K - 1].real
    A = np.vstack([rows, math.sqrt(lam) * np.eye(K)])
    y = np.concatenate([np.sqrt(w[nz]) * G[nz], np.zeros(K)])
    rho_ls = np.linalg.lstsq(A, y, rcond=None)[0]
    assert np.linalg.norm(out["taps"] - rho_ls) <= 1e-7 * np.linalg.norm(rho_ls)


def test_closed_form_match_equals_fft_match(S):
    tmpl = (1.43, 1.38, 0.0, 0.0, 0.0)
    out = fit.design(FS, N, FLOW, tmpl, REF, S, 64, 1e-6)
    h_ref = wf.template(FS, N, FLOW, REF)
    h_j = wf.template(FS, N, FLOW, tmpl)
    m = ratio.tap_match(h_j, out["taps"], out["lag"], h_ref, S, DF, N)
    assert abs(out["match"] - m) < 1e-10
    s2 = ratio.sigma_eff_sq_freq(out["taps"], out["lag"], h_ref, S, DF, N)
    assert abs(out["sigma_eff"] ** 2 / s2 - 1) < 1e-10


def test_identity_template_is_fitted_by_minimum_norm_taps(S):
    K = 32
    out = fit.design(FS, N, FLOW, REF, REF, S, K, 1e-12)
    assert out["lag"] == -K // 2
    assert out["match"] > 1 - 1e-10
    G = ratio.ratio_spectrum(FS, N, FLOW, REF, REF)
    w = fit.weights(wf.template(FS, N, FLOW, REF), S, DF)
    assert chi2(out["taps"], G, w, out["lag"], 0.0) < 1e-8 * float(np.sum(w))
    assert np.linalg.norm(out["taps"]) < 1.0          # the delta at -s has norm 1


def test_fit_beats_windowed_taps(S):
    for tmpl in [(1.45, 1.40, 0.0, 0.0, 0.0), (1.50, 1.36, 0.0, 0.0, 0.0), (1.38, 1.37, 0.0, 0.0, 0.0)]:
        K = 48
        f = fit.design(FS, N, FLOW, tmpl, REF, S, K, 1e-6)
        w = ratio.design(FS, N, FLOW, tmpl, REF, S, K)
        assert f["lag"] == w["lag"]
        assert f["match"] >= w["match"] - 1e-12
    assert f["match"] > w["match"]


def test_ridge_shrinks_taps(S):
    tmpl = (1.45, 1.40, 0.0, 0.0, 0.0)
    K = 48
    G = ratio.ratio_spectrum(FS, N, FLOW, tmpl, REF)
    w = fit.weights(wf.template(FS, N, FLOW, REF), S, DF)
    prev_norm, prev_chi = None, None
    for eps in (1e-8, 1e-5, 1e-3, 1e-1):
        out = fit.design(FS, N, FLOW, tmpl, REF, S, K, eps)
        nrm = np.linalg.norm(out["taps"])
        c = chi2(out["taps"], G, w, out["lag"], 0.0)
        if prev_norm is not None:
            assert nrm <= prev_norm * (1 + 1e-9)
            assert c >= prev_chi * (1 - 1e-9)
        prev_norm, prev_chi = nrm, c


def test_dynamic_k_is_smallest_bucket_reaching_target(S):
    tmpl = (1.41, 1.40, 0.0, 0.0, 0.0)
    buckets = [16, 32, 64, 128]
    target = 0.99
    out = fit.design_dynamic(FS, N, FLOW, tmpl, REF, S, buckets, target)
    assert out["match"] >= target
    smaller = [b for b in buckets if b < out["K"]]
    for b in smaller:
        assert fit.design(FS, N, FLOW, tmpl, REF, S, b)["match"] < target

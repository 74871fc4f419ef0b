"""Pins for the oracle's learned-tap network (oracle/mlp.py).

* GELU: the tanh form satisfies gelu(u) - gelu(-u) = u exactly and stays within 1e-3 of the
  erf form u Phi(u) (its published approximation); its derivative matches central
  differences;
* loss: zero at the target and at any phase rotation of it, 1 for twice the target, the
  orthogonal closed form, and 2 (1 - match) for equal norms with the match computed in the
  frequency domain; the quadratic form equals the frequency-domain chi^2 of Eq. 4 / Eq. 5
  computed through the FFT of the placed taps (Parseval, an independent path);
* phasor inputs: all cos = 1, sin = 0 for the reference itself, and equal to the phase of the
  ratio spectrum G of Eq. 2 (ratio.ratio_spectrum) at grid frequencies;
* cross match: 1 for a tap set against itself or a phase rotation of it, and equal to the
  frequency-domain overlap of the two effective templates;
* backward: every gradient tensor agrees with central finite differences of the loss, both
  on sampled entries and along a random direction in the whole parameter space;
* Adam: a constant gradient gives the closed-form step lr g / (|g| + eps) at every t;
* features: closed forms for equal masses and for chi_eff.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import workload
from oracle import mlp, ratio, waveform as wf

FS, N, FLOW = 256.0, 4096, 20.0
DF = FS / N
K = mlp.K_TAPS


def psd_grid():
    f = np.arange(N // 2 + 1) * DF
    S = np.empty(N // 2 + 1)
    S[1:] = workload.psd_analytic(f[1:])
    S[0] = S[1]
    return S


@pytest.fixture(scope="module")
def ref_C():
    S = psd_grid()
    h_ref = wf.template(FS, N, FLOW, (1.4, 1.4, 0, 0, 0))
    C = ratio.autocorrelation(h_ref, S, DF, N, K - 1)
    return h_ref, S, C


def small_net(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W, b = [], []
    for (o, i) in mlp.init_shapes():
        W.append(rng.uniform(-1, 1, (o, i)) * scale / math.sqrt(i))
        b.append(rng.uniform(-0.1, 0.1, o))
    return W, b


def test_gelu_odd_part_and_erf_form():
    u = np.linspace(-8, 8, 4001)
    assert np.max(np.abs(mlp.gelu(u) - mlp.gelu(-u) - u)) < 1e-14
    exact = 0.5 * u * (1.0 + erf(u / math.sqrt(2.0)))
    assert np.max(np.abs(mlp.gelu(u) - exact)) < 1e-3
    h = 1e-6
    fd = (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(u))) < 1e-8


def test_loss_closed_forms(ref_C):
    h_ref, S, C = ref_C
    rng = np.random.default_rng(1)
    a = rng.standard_normal((3, K)) + 1j * rng.standard_normal((3, K))
    loss, g = mlp.loss_and_grad_taps(a.copy(), a, C)
    assert abs(loss) < 1e-13 and np.max(np.abs(g)) < 1e-12 * np.max(np.abs(a))
    for phi in (0.1, 1.0, 2.5):
        loss, _ = mlp.loss_and_grad_taps(a * np.exp(1j * phi), a, C)
        assert abs(loss) < 1e-12
    loss, _ = mlp.loss_and_grad_taps(2 * a, a, C)
    assert abs(loss - 1.0) < 1e-12
    # a tap set orthogonal to the target under M: L = (s_rho + s_a) / s_a
    M = mlp.toeplitz_c(C)
    x = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    u = M @ a[0]
    x = x - (np.vdot(u, x) / np.vdot(u, a[0])) * a[0]           # a^H M x = 0
    s_x = np.real(np.vdot(x, M @ x))
    s_a = np.real(np.vdot(a[0], M @ a[0]))
    loss, _ = mlp.loss_and_grad_taps(x[None], a[:1], C)
    assert abs(loss - (s_x + s_a) / s_a) < 1e-10
    # equal norms: L = 2 (1 - match), the match taken in the frequency domain
    r = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    r *= math.sqrt(s_a / np.real(np.vdot(r, M @ r)))
    loss, _ = mlp.loss_and_grad_taps(r[None], a[:1], C)
    s = -K // 2
    A1 = ratio.effective_response(r, s, N)[: N // 2 + 1]
    A2 = ratio.effective_response(a[0], s, N)[: N // 2 + 1]
    nz = np.nonzero(h_ref)[0]
    wgt = np.abs(h_ref[nz]) ** 2 / S[nz]
    match = abs(np.sum(wgt * A1[nz] * np.conj(A2[nz]))) / math.sqrt(
        np.sum(wgt * np.abs(A1[nz]) ** 2) * np.sum(wgt * np.abs(A2[nz]) ** 2))
    assert abs(loss - 2 * (1 - match)) < 1e-10


def test_phasor_inputs():
    ref = (1.4, 1.35, 0.01, -0.02, 300.0)
    ph = mlp.phasor_features([ref], ref, FS, FLOW, wf.PN_TIDAL)
    assert np.all(ph[0, :mlp.N_PHASOR] == 1.0) and np.all(ph[0, mlp.N_PHASOR:] == 0.0)
    # at grid frequencies the phasors are the phase of G = exp(+i (Psi_j - Psi_r)) (Eq. 2)
    tmpl = (1.43, 1.33, 0.02, 0.0, 900.0)
    G = ratio.ratio_spectrum(FS, N, FLOW, tmpl, ref, wf.PN_TIDAL)
    f = mlp.phasor_frequencies(FS, FLOW)
    k = np.rint(f / DF).astype(int)
    orig = mlp.phasor_frequencies
    try:
        mlp.phasor_frequencies = lambda fs, fl: k * DF
        got = mlp.phasor_features([tmpl], ref, FS, FLOW, wf.PN_TIDAL)[0]
    finally:
        mlp.phasor_frequencies = orig
    want = np.delete(G[k] * np.conj(G[k[mlp.N_PHASOR // 2]]), mlp.N_PHASOR // 2)
    assert np.allclose(got[:mlp.N_PHASOR], want.real, atol=1e-9)
    assert np.allclose(got[mlp.N_PHASOR:], want.imag, atol=1e-9)
    x = mlp.network_inputs([tmpl], ref, np.zeros(4), np.ones(4), FS, FLOW, wf.PN_TIDAL)
    assert x.shape == (1, mlp.N_FEAT) == (1, 20)


def test_loss_numerator_is_frequency_domain_chi2(ref_C):
    h_ref, S, C = ref_C
    rng = np.random.default_rng(2)
    d = rng.standard_normal(K) + 1j * rng.standard_normal(K)
    M = mlp.toeplitz_c(C)
    quad = float(np.real(np.conj(d) @ (M @ d)))
    freq = ratio.sigma_eff_sq_freq(d, -K // 2, h_ref, S, DF, N)
    assert abs(quad / freq - 1) < 1e-11


def test_cross_match(ref_C):
    h_ref, S, C = ref_C
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, K)) + 1j * rng.standard_normal((2, K))
    assert np.allclose(mlp.cross_match(a, a, C), 1.0, atol=1e-13)
    assert np.allclose(mlp.cross_match(a * np.exp(0.7j), a, C), 1.0, atol=1e-13)
    s = -K // 2
    got = mlp.cross_match(a[:1], a[1:], C)[0]
    A1 = ratio.effective_response(a[0], s, N)[: N // 2 + 1]
    A2 = ratio.effective_response(a[1], s, N)[: N // 2 + 1]
    nz = np.nonzero(h_ref)[0]
    wgt = np.abs(h_ref[nz]) ** 2 / S[nz]
    e1, e2 = h_ref[nz] * np.conj(A1[nz]), h_ref[nz] * np.conj(A2[nz])
    x = np.sum(np.conj(e2) * e1 / S[nz])
    want = abs(x) / math.sqrt(np.sum(np.abs(A1[nz]) ** 2 * wgt) * np.sum(np.abs(A2[nz]) ** 2 * wgt))
    assert abs(got - want) < 1e-11


def _loss(W, b, xh, target, C, scale):
    y, _ = mlp.forward(W, b, xh)
    return mlp.loss_and_grad_taps(mlp.taps_from_output(y, scale), target, C)[0]


def test_backward_against_finite_differences(ref_C):
    _, _, C = ref_C
    W, b = small_net(4)
    rng = np.random.default_rng(5)
    B = 6
    xh = rng.standard_normal((B, mlp.N_FEAT))
    target = 0.05 * (rng.standard_normal((B, K)) + 1j * rng.standard_normal((B, K)))
    scale = 0.03
    loss, dW, db = mlp.loss_and_grads(W, b, xh, target, C, scale)
    assert loss == pytest.approx(_loss(W, b, xh, target, C, scale), rel=1e-14)
    h = 1e-6
    for l in range(mlp.N_LAYERS):
        for (P, G) in ((W[l], dW[l]), (b[l], db[l])):
            flat = P.reshape(-1)
            gflat = G.reshape(-1)
            for idx in rng.choice(flat.size, size=12, replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = _loss(W, b, xh, target, C, scale)
                flat[idx] = old - h
                lm = _loss(W, b, xh, target, C, scale)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                # relative 1e-6, above the difference quotient's own rounding floor (~eps L / h)
                assert abs(fd - gflat[idx]) <= 1e-6 * abs(fd) + 1e-9 * max(1.0, loss), (l, idx)
    # directional derivative over all parameters at once
    vW = [rng.standard_normal(w.shape) for w in W]
    vb = [rng.standard_normal(x.shape) for x in b]
    eps = 1e-6
    lp = _loss([w + eps * v for w, v in zip(W, vW)], [x + eps * v for x, v in zip(b, vb)], xh, target, C, scale)
    lm = _loss([w - eps * v for w, v in zip(W, vW)], [x - eps * v for x, v in zip(b, vb)], xh, target, C, scale)
    want = sum(np.sum(g * v) for g, v in zip(dW, vW)) + sum(np.sum(g * v) for g, v in zip(db, vb))
    assert abs((lp - lm) / (2 * eps) / want - 1) < 1e-6


def test_adam_constant_gradient_closed_form():
    rng = np.random.default_rng(6)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        p_new, m, v = mlp.adam_step(p, g, m, v, t, lr, eps=eps)
        assert np.allclose(p - p_new, lr * g / (np.abs(g) + eps), rtol=1e-9, atol=0)
        p = p_new


def test_features_closed_forms():
    f = mlp.features([(1.4, 1.4, 0.1, -0.1, 300.0), (2.0, 1.0, 0.2, 0.4, 0.0)])
    assert f[0, 1] == pytest.approx(0.25, rel=1e-15)
    assert f[0, 0] == pytest.approx(2.8 / 2 ** 1.2, rel=1e-14)
    assert f[0, 2] == pytest.approx(0.0, abs=1e-15)
    assert f[0, 3] == 300.0
    assert f[1, 1] == pytest.approx(2.0 / 9.0, rel=1e-15)
    assert f[1, 0] == pytest.approx((2.0 * 1.0) ** 0.6 / 3.0 ** 0.2, rel=1e-14)
    assert f[1, 2] == pytest.approx((2 * 0.2 + 0.4) / 3, rel=1e-14)

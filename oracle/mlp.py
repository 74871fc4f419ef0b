"""Learned taps: a small MLP from template parameters to ratio-filter taps, in FP64 (oracle;
test infrastructure).

Sec. V.A builds each template's taps by minimising the PSD-weighted chi^2 of Eq. 4 between
the taps' frequency response and the ratio.  The surrogate here learns the map from the
template's physical parameters to those taps, one network per reference, so that a new
template's taps cost one forward pass instead of an N-point transform.  The paper's closing
discussion (Sec. VI) notes the compact ratio kernel as a bridge to ML pipelines; the network
itself is this implementation's design, and every piece of it is written out below.

Inputs (per template j of reference r): the physical features x = (Mc, eta, chi_eff, Lambda~),
standardised per network, xh = (x - mu_r) / sd_r, followed by eight phasors of the ratio's own
phase (Eq. 2): with Dpsi(f) = Psi_j(f) - Psi_r(f) and nine frequencies f_0..f_8 log-spaced from
3 f_low to 0.45 fs, the anchor f_a = f_4 and
  p_m = Dpsi(f_m) - Dpsi(f_a),   inputs cos p_m, sin p_m   (m != 4),
20 inputs in all.  The taps turn through many radians across one reference's group, and the
phasors hand the network that rotation directly.

Network (per reference r):
  h1 = gelu(W1 in + b1),  h2 = gelu(W2 h1 + b2),  h3 = gelu(W3 h2 + b3)       (256 wide)
  y  = W4 h3 + b4                                                          (256 = 2 x 128)
  rho[k] = out_scale_r (y[k] + i y[128 + k]),  k < 128, taps at the reference's fixed lag s_r
  gelu(u) = u/2 (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3)))   (tanh form, Hendrycks & Gimpel)

Loss (per sample, mean over the batch): the chi^2 of Eq. 4 between the taps' response and the
exact taps' response, weighted by |h_ref|^2 / S and written in the tap domain through Parseval
(Eqs. 5-6), minimised over a constant phase of the target (a constant phase of a template's
taps only rotates its complex SNR, which the search maximises over):
  L = min_phi (rho - e^{i phi} a*)^H M (rho - e^{i phi} a*) / (a*^H M a*)
    = (rho^H M rho + a*^H M a* - 2 |a*^H M rho|) / (a*^H M a*),     M[b, a] = C_r[b - a]
with C_r the reference autocorrelation on the sample grid (ratio.autocorrelation) and a* the
exact taps at the same lag.  For equal norms L = 2 (1 - match).

Surrogate check: the match between the responses of two tap sets placed at the same lag,
  |sum_{a,b} rho1[a] conj(rho2[b]) C_r[b - a]| / (sigma1 sigma2).

Adam (Kingma & Ba 2015, bias-corrected) updates the FP32 master weights on the GPU; adam_step
below is its FP64 statement.
"""
import math

import numpy as np

from . import waveform as _wf

N_HIDDEN = 256
N_LAYERS = 4            # three hidden layers + the output layer
N_PHYS = 4
N_PHASOR = 8
N_FEAT = N_PHYS + 2 * N_PHASOR
K_TAPS = 128
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


# ---------------------------------------------------------------- features
def features(params):
    """(Mc, eta, chi_eff, Lambda~) of each template; params rows (m1, m2, chi1, chi2, lam)."""
    p = np.asarray(params, dtype=np.float64).reshape(-1, 5)
    m1, m2, c1, c2, lam = p.T
    M = m1 + m2
    eta = m1 * m2 / M ** 2
    mc = M * eta ** 0.6
    chi_eff = (m1 * c1 + m2 * c2) / M
    return np.stack([mc, eta, chi_eff, lam], axis=1)


def phasor_frequencies(fs, f_low):
    """Nine frequencies log-spaced from 3 f_low to 0.45 fs; the middle one is the anchor."""
    return np.geomspace(3.0 * f_low, 0.45 * fs, N_PHASOR + 1)


def phasor_features(params, ref_params, fs, f_low, pn_flags=0):
    """cos and sin of Dpsi(f_m) - Dpsi(f_a) for the eight non-anchor frequencies."""
    f = phasor_frequencies(fs, f_low)
    r = np.asarray(ref_params, dtype=np.float64)
    psi_r = _wf.phase(f, r[0], r[1], r[2], r[3], r[4], pn_flags)
    out = []
    for p in np.asarray(params, dtype=np.float64).reshape(-1, 5):
        dpsi = _wf.phase(f, p[0], p[1], p[2], p[3], p[4], pn_flags) - psi_r
        ph = np.delete(dpsi - dpsi[N_PHASOR // 2], N_PHASOR // 2)
        out.append(np.concatenate([np.cos(ph), np.sin(ph)]))
    return np.array(out).reshape(-1, 2 * N_PHASOR)


def network_inputs(params, ref_params, mu, sd, fs, f_low, pn_flags=0):
    """The 20 inputs of one network: standardised physical features, then the phasors."""
    xh = (features(params) - mu) / sd
    return np.concatenate([xh, phasor_features(params, ref_params, fs, f_low, pn_flags)], axis=1)


def standardiser(x):
    """Mean and spread of a training set's features; a constant feature keeps spread 1."""
    mu = x.mean(axis=0)
    sd = x.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return mu, sd


# ---------------------------------------------------------------- GELU
def gelu(u):
    return 0.5 * u * (1.0 + np.tanh(GELU_C * (u + GELU_A * u ** 3)))


def gelu_grad(u):
    t = np.tanh(GELU_C * (u + GELU_A * u ** 3))
    return 0.5 * (1.0 + t) + 0.5 * u * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * u * u)


# ---------------------------------------------------------------- one network
def forward(W, b, xh):
    """W[l]: (out, in), b[l]: (out,); xh: (B, 20) network inputs.  Returns y (B, 256) and the cache
    (inputs and pre-activations of every layer) the backward pass needs."""
    h = xh
    cache = []
    for l in range(N_LAYERS):
        z = h @ W[l].T + b[l]
        cache.append((h, z))
        h = gelu(z) if l < N_LAYERS - 1 else z
    return h, cache


def taps_from_output(y, out_scale):
    return out_scale * (y[:, :K_TAPS] + 1j * y[:, K_TAPS:])


def toeplitz_c(C, K=K_TAPS):
    """M[b, a] = C[b - a] from C[l], l = -(K-1) .. K-1 stored at index l + K - 1."""
    mid = (len(C) - 1) // 2
    i = np.arange(K)
    return C[mid + i[:, None] - i[None, :]]


def loss_and_grad_taps(rho, target, C):
    """Mean phase-minimised chi^2 over the batch and its gradient with respect to
    (Re rho, Im rho), returned as d loss / d Re rho + i d loss / d Im rho.
    rho, target: (B, K) complex.  With c = a*^H M rho the minimising phase is arg c, and the
    gradient is that of the plain chi^2 against the rotated target e^{i arg c} a*."""
    M = toeplitz_c(C, rho.shape[1])
    Mr = rho @ M.T                                  # (M rho)[b] = sum_a M[b, a] rho[a]
    Mt = target @ M.T
    s_r = np.real(np.sum(np.conj(rho) * Mr, axis=1))
    s_t = np.real(np.sum(np.conj(target) * Mt, axis=1))
    c = np.sum(np.conj(Mt) * rho, axis=1)           # a*^H M rho (M Hermitian)
    B = rho.shape[0]
    loss = float(np.mean((s_r + s_t - 2.0 * np.abs(c)) / s_t))
    ph = np.where(np.abs(c) > 0, c / np.where(np.abs(c) > 0, np.abs(c), 1.0), 1.0)
    g = 2.0 * (Mr - ph[:, None] * Mt) / s_t[:, None] / B
    return loss, g


def backward(W, cache, dy):
    """Gradients of every weight and bias given d loss / d y (B, 256)."""
    dW = [None] * N_LAYERS
    db = [None] * N_LAYERS
    g = dy
    for l in range(N_LAYERS - 1, -1, -1):
        h_in, z = cache[l]
        if l < N_LAYERS - 1:
            g = g * gelu_grad(z)
        dW[l] = g.T @ h_in
        db[l] = g.sum(axis=0)
        g = g @ W[l]
    return dW, db


def loss_and_grads(W, b, xh, target, C, out_scale):
    """Loss and parameter gradients for one batch of one network."""
    y, cache = forward(W, b, xh)
    rho = taps_from_output(y, out_scale)
    loss, g = loss_and_grad_taps(rho, target, C)
    dy = out_scale * np.concatenate([g.real, g.imag], axis=1)
    dW, db = backward(W, cache, dy)
    return loss, dW, db


def init_shapes():
    return [(N_HIDDEN, N_FEAT)] + [(N_HIDDEN, N_HIDDEN)] * (N_LAYERS - 1)


# ---------------------------------------------------------------- Adam
def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma & Ba 2015, Algorithm 1); returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- surrogate check
def cross_match(rho1, rho2, C):
    """Match between the responses of two tap sets at the same lag (rows of rho1, rho2)."""
    M = toeplitz_c(C, rho1.shape[1])
    x12 = np.sum(np.conj(rho2) * (rho1 @ M.T), axis=1)
    s1 = np.real(np.sum(np.conj(rho1) * (rho1 @ M.T), axis=1))
    s2 = np.real(np.sum(np.conj(rho2) * (rho2 @ M.T), axis=1))
    return np.abs(x12) / np.sqrt(s1 * s2)

"""Learned taps on the GPU (librfd's MLP kernels) against the FP64 oracle.

* the references' autocorrelations C_r and the fixed-lag taps (rfd_make_taps_at_lag) equal
  the oracle's;
* the FP16 network inputs, the forward pass (rfd_mlp_infer) and sigma_eff of the output taps
  equal the oracle's on the same weights;
* the gradients of every weight and bias (rfd_mlp_grads) equal the oracle's backward pass on
  the same weights and batch (relative error <= 1e-2 per tensor, cosine >= 0.999);
* one optimiser step (rfd_mlp_train_step) equals the oracle's Adam statement applied to the
  same gradients;
* trained on oracle-generated tap sets in the dense-reference regime, the networks reach the
  0.999 surrogate match on held-out templates, and rfd_learned_taps keeps their taps there,
  so that most templates skip exact extraction (the gain over taps from make_taps alone).
"""
import math
import time

import numpy as np
import pytest

import workload
from oracle import mlp, ratio
from tests import oracle_mlp_data as omd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402

FS, N, FLOW = 2048.0, 32768, 20.0
PN = workload.configs.PN_TIDAL
K = 128
REFS = np.array([[1.45, 1.35, 0.0, 0.0, 700.0], [1.25, 1.18, 0.01, -0.01, 300.0]])
DELTA = 0.002
N_TRAIN, N_HELD = 6144, 256


@pytest.fixture(scope="module")
def env():
    cfg = workload.small_config(4, n=N, n_tmpl=4, n_ref=1, n_inj=0)
    _, data = workload.make_workload(cfg)
    ctx = rfd.Context(0)
    g = rfd.grid(FS, N, FLOW, PN)
    psd = torch.from_numpy(data.psd).cuda()
    net = rfd.Mlp(ctx, g, psd, REFS)
    C = omd.autocorr(FS, N, FLOW, PN, REFS, data.psd)
    yield {"ctx": ctx, "g": g, "psd": psd, "psd_np": data.psd, "mlp": net, "C": C}
    net.close()


@pytest.fixture(scope="module")
def dense(env):
    """Oracle-generated training and held-out sets, per reference, at the references' lags."""
    train = workload.dense_bank(REFS, N_TRAIN, DELTA, seed=41)
    held = workload.dense_bank(REFS, N_HELD, DELTA, seed=42)
    P, ro = train.params(), train.ref_of_tmpl
    sample = np.concatenate([np.nonzero(ro == r)[0][:64] for r in range(len(REFS))])
    lags_own = omd.own_lags(FS, N, FLOW, PN, P[sample], REFS, ro[sample])
    lag = np.array([int(np.median(lags_own[ro[sample] == r])) for r in range(len(REFS))], dtype=np.int32)
    T = omd.targets(FS, N, FLOW, PN, P, REFS, ro, lag)
    Th = omd.targets(FS, N, FLOW, PN, held.params(), REFS, held.ref_of_tmpl, lag)
    feats = mlp.features(P)
    mu = np.stack([mlp.standardiser(feats[ro == r])[0] for r in range(len(REFS))])
    sd = np.stack([mlp.standardiser(feats[ro == r])[1] for r in range(len(REFS))])
    scale = np.array([math.sqrt(np.mean(np.abs(T[ro == r]) ** 2)) for r in range(len(REFS))])
    return {"train": train, "held": held, "lag": lag, "T": T, "Th": Th, "mu": mu, "sd": sd, "scale": scale}


def _set_norm(env, dense):
    env["mlp"].set_norm(dense["mu"], dense["sd"], dense["scale"], dense["lag"])


def test_autocorr_matches_oracle(env):
    got = env["mlp"].autocorr()
    want = env["C"]
    for r in range(len(REFS)):
        assert np.max(np.abs(got[r] - want[r])) <= 1e-9 * abs(want[r][K - 1])


def test_make_taps_at_lag_matches_oracle(env):
    bank = workload.dense_bank(REFS, 6, 0.01, seed=3)
    P, ro = bank.params(), bank.ref_of_tmpl
    lags = np.array([-64, -100, 30, -1, -128, 5, -64, -20, 17, -90, 0, -127], dtype=np.int32)
    Kj = np.full(len(P), K, dtype=np.int32)
    taps = torch.zeros((len(P), K), dtype=torch.complex64, device="cuda")
    sig = torch.zeros(len(P), dtype=torch.float64, device="cuda")
    rfd.make_taps_at_lag(env["ctx"], env["g"], env["psd"], REFS, P, ro, Kj, lags, K, 0.1, taps, sig)
    torch.cuda.synchronize()
    t = taps.cpu().numpy()
    s = sig.cpu().numpy()
    for j in range(len(P)):
        g = ratio.impulse_response(ratio.ratio_spectrum(FS, N, FLOW, P[j], REFS[ro[j]], PN))
        want = ratio.taps_at_lag(g, K, 0.1, int(lags[j]))
        assert np.max(np.abs(t[j] - want)) <= 2e-7 * np.max(np.abs(want)) + 1e-12
        s2 = ratio.sigma_eff_sq_parseval(want, env["C"][ro[j]])
        assert abs(s[j] / math.sqrt(s2) - 1) < 1e-9


def test_inputs_match_oracle(env, dense):
    _set_norm(env, dense)
    held = dense["held"]
    P, ro = held.params()[:200], held.ref_of_tmpl[:200]
    got = env["mlp"].features(P, ro).float().cpu().numpy()
    want = omd.inputs(FS, FLOW, PN, P, REFS, ro, dense["mu"], dense["sd"])
    assert np.all(got[:, mlp.N_FEAT:] == 0)
    assert np.max(np.abs(got[:, :mlp.N_FEAT] - want)) <= 2e-3 * max(1.0, np.max(np.abs(want)))


def _oracle_forward(w_flat, x16, scale):
    """The oracle's forward pass on the FP16-rounded weights and inputs the GPU uses."""
    W, b = omd.unflatten(w_flat)
    W = [w.astype(np.float16).astype(np.float64) for w in W]
    y, _ = mlp.forward(W, b, x16)
    return mlp.taps_from_output(y, scale)


def test_forward_matches_oracle(env, dense):
    _set_norm(env, dense)
    w = omd.init_weights(len(REFS), seed=5)
    env["mlp"].set_weights(w)
    held = dense["held"]
    sel = np.arange(0, held.n_tmpl, 3)
    P, ro = held.params()[sel], held.ref_of_tmpl[sel]
    taps = torch.zeros((len(P), 160), dtype=torch.complex64, device="cuda")
    lag = torch.zeros(len(P), dtype=torch.int32, device="cuda")
    sig = torch.zeros(len(P), dtype=torch.float64, device="cuda")
    env["mlp"].infer(P, ro, taps, lag, sig)
    t = taps.cpu().numpy()
    assert np.all(t[:, K:] == 0)
    assert np.array_equal(lag.cpu().numpy(), dense["lag"][ro])
    x16 = env["mlp"].features(P, ro).float().cpu().numpy()[:, :mlp.N_FEAT].astype(np.float64)
    s = sig.cpu().numpy()
    for r in range(len(REFS)):
        m = ro == r
        want = _oracle_forward(w[r], x16[m], dense["scale"][r])
        err = np.linalg.norm(t[m, :K] - want, axis=1) / np.linalg.norm(want, axis=1)
        assert np.max(err) < 1e-2, np.max(err)
        s_want = np.sqrt([ratio.sigma_eff_sq_parseval(x.astype(np.complex128), env["C"][r]) for x in t[m, :K]])
        assert np.max(np.abs(s[m] / s_want - 1)) < 1e-6


def _batch(dense, B, seed):
    rng = np.random.default_rng(seed)
    return np.stack([rng.choice(N_TRAIN, B, replace=False) for _ in REFS]).astype(np.int32)


def _train_tensors(env, dense):
    train = dense["train"]
    P, ro = train.params(), train.ref_of_tmpl
    order = np.argsort(ro, kind="stable")        # rows grouped by network: [R][N_TRAIN]
    feat = env["mlp"].features(P[order], ro[order])
    tgt = torch.from_numpy(dense["T"][order].astype(np.complex64)).cuda()
    return feat, tgt, order


def test_grads_match_oracle(env, dense):
    _set_norm(env, dense)
    w = omd.init_weights(len(REFS), seed=6)
    env["mlp"].set_weights(w)
    feat, tgt, order = _train_tensors(env, dense)
    B = 256
    idx = _batch(dense, B, seed=7)
    grads, loss = env["mlp"].grads(feat, tgt, N_TRAIN, torch.from_numpy(idx).cuda(), B)
    grads = grads.cpu().numpy().astype(np.float64)
    loss = loss.cpu().numpy()
    x16 = feat.float().cpu().numpy()[:, :mlp.N_FEAT].astype(np.float64)
    T = dense["T"][order]
    for r in range(len(REFS)):
        rows = r * N_TRAIN + idx[r]
        W, b = omd.unflatten(w[r])
        W = [x.astype(np.float16).astype(np.float64) for x in W]
        l_ora, dW, db = mlp.loss_and_grads(W, b, x16[rows], T[rows], env["C"][r], dense["scale"][r])
        assert abs(loss[r] / l_ora - 1) < 2e-3, (loss[r], l_ora)
        gW, gb = omd.unflatten(grads[r])
        for name, got, want in [("W%d" % l, gW[l], dW[l]) for l in range(4)] + \
                               [("b%d" % l, gb[l], db[l]) for l in range(4)]:
            rel = np.linalg.norm(got - want) / np.linalg.norm(want)
            cos = np.sum(got * want) / (np.linalg.norm(got) * np.linalg.norm(want))
            assert rel <= 1e-2 and cos >= 0.999, (r, name, rel, cos)


def test_adam_step_matches_oracle(env, dense):
    _set_norm(env, dense)
    w = omd.init_weights(len(REFS), seed=8)
    env["mlp"].set_weights(w)
    feat, tgt, _ = _train_tensors(env, dense)
    B = 128
    idx = torch.from_numpy(_batch(dense, B, seed=9)).cuda()
    grads, _ = env["mlp"].grads(feat, tgt, N_TRAIN, idx, B)
    lr = 1e-3
    env["mlp"].train_step(feat, tgt, N_TRAIN, idx, B, lr)
    _, step, _ = env["mlp"].state()
    assert step == 1
    got = env["mlp"].get_weights().astype(np.float64)
    g = grads.cpu().numpy().astype(np.float64)
    want, _, _ = mlp.adam_step(w.astype(np.float64), g, 0.0, 0.0, 1, lr)
    assert np.max(np.abs(got - want)) <= 1e-6 * max(1.0, np.max(np.abs(w))) + 1e-3 * lr


def test_training_reaches_target_and_learned_taps_gain(env, dense):
    net = env["mlp"]
    _set_norm(env, dense)
    net.set_weights(omd.init_weights(len(REFS), seed=10))
    feat, tgt, _ = _train_tensors(env, dense)
    B, epochs, lr0 = 256, 300, 3e-3
    steps_per_epoch = N_TRAIN // B
    rng = np.random.default_rng(11)
    idx_all = np.stack([np.stack([rng.permutation(N_TRAIN)[:steps_per_epoch * B].reshape(steps_per_epoch, B)
                                  for _ in REFS], axis=1) for _ in range(epochs)]).reshape(-1, len(REFS), B)
    idx_dev = torch.from_numpy(idx_all.astype(np.int32)).cuda()
    grads0, loss0 = net.grads(feat, tgt, N_TRAIN, idx_dev[0].contiguous(), B)
    t0 = time.time()
    n_steps = idx_all.shape[0]
    for s in range(n_steps):
        lr = lr0 * 0.5 * (1 + math.cos(math.pi * (s // steps_per_epoch) / epochs))
        net.train_step(feat, tgt, N_TRAIN, idx_dev[s], B, max(lr, 1e-6))
    loss, steps, scale = net.state()
    t_train = time.time() - t0
    assert steps >= n_steps - 20                 # a few steps may be skipped by the loss scaling
    assert np.all(loss < loss0.cpu().numpy() / 20), (loss, loss0)
    # held-out surrogate match against the oracle's exact taps at the same lag
    held = dense["held"]
    P, ro = held.params(), held.ref_of_tmpl
    taps = torch.zeros((len(P), K), dtype=torch.complex64, device="cuda")
    lag = torch.zeros(len(P), dtype=torch.int32, device="cuda")
    sig = torch.zeros(len(P), dtype=torch.float64, device="cuda")
    net.infer(P, ro, taps, lag, sig)
    t = taps.cpu().numpy().astype(np.complex128)
    m = np.empty(len(P))
    for r in range(len(REFS)):
        sel = ro == r
        m[sel] = mlp.cross_match(t[sel], dense["Th"][sel], env["C"][r])
    # the library's own match kernel agrees with the oracle's
    exact = torch.from_numpy(dense["Th"].astype(np.complex64)).cuda()
    m_gpu = net.cross_match(ro, taps, exact).cpu().numpy()
    assert np.max(np.abs(m_gpu - m)) < 1e-6
    frac = float(np.mean(m >= 0.999))
    print("train %.2fs, final loss %s, held-out match median %.5f, >=0.999: %.3f" % (t_train, loss, np.median(m), frac))
    assert np.median(m) >= 0.998 and frac >= 0.5
    # surrogate with spot checks and exact fallback
    out = torch.zeros((len(P), K), dtype=torch.complex64, device="cuda")
    lag2 = torch.zeros(len(P), dtype=torch.int32, device="cuda")
    sig2 = torch.zeros(len(P), dtype=torch.float64, device="cuda")
    source, smatch, stats = net.learned_taps(env["psd"], P, ro, out, lag2, sig2, spot_stride=8, min_match=0.999)
    src = source.cpu().numpy()
    assert stats["surrogate"] + stats["exact"] == len(P)
    assert stats["surrogate"] == int(np.sum(src != 1)) and stats["exact"] == int(np.sum(src == 1))
    sm = smatch.cpu().numpy()
    spot = ~np.isnan(sm)
    assert int(spot.sum()) == stats["spot_checked"]
    assert np.allclose(sm[spot], m[spot], atol=1e-6)           # the spot matches are the held-out matches
    # surrogate templates carry the network's taps; fallback templates the exact own-lag taps
    o = out.cpu().numpy()
    keep = src != 1
    assert np.array_equal(o[keep], taps.cpu().numpy()[keep])
    assert np.min(m[keep]) >= 0.995
    fb = np.nonzero(src == 1)[0][:6]
    for j in fb:
        d = ratio.design(FS, N, FLOW, P[j], REFS[ro[j]], env["psd_np"], K, 0.1, PN, with_match=False)
        assert int(lag2[j]) == d["lag"]
        assert np.max(np.abs(o[j] - d["taps"])) <= 2e-7 * np.max(np.abs(d["taps"])) + 1e-12
    extractions = stats["spot_checked"] + stats["exact"]
    print("learned taps: %s; exact extractions %d of %d" % (stats, extractions, len(P)))
    assert extractions < 0.5 * len(P)


def test_checkpoint_resume_is_bit_exact(env, dense, tmp_path):
    """rfd_mlp_save / rfd_mlp_load: N optimiser steps, a checkpoint, a fresh network object
    that loads it, M more steps gives the same master weights, Adam state and loss scale, bit
    for bit, as N + M steps without the interruption.  A checkpoint made for other
    references is refused."""
    from paper_2601_18835_gb300 import _native
    _set_norm(env, dense)
    w0 = omd.init_weights(len(REFS), seed=21)
    feat, tgt, _ = _train_tensors(env, dense)
    B, n1, n2 = 128, 12, 9
    rng = np.random.default_rng(22)
    idx = torch.from_numpy(np.stack([np.stack([rng.permutation(N_TRAIN)[:B] for _ in REFS])
                                     for _ in range(n1 + n2)]).astype(np.int32)).cuda()
    lrs = [3e-3 * (0.9 ** s) for s in range(n1 + n2)]

    def run(net, steps):
        for s in steps:
            net.train_step(feat, tgt, N_TRAIN, idx[s].contiguous(), B, lrs[s])
        torch.cuda.synchronize()

    ref = env["mlp"]
    ref.set_weights(w0)
    run(ref, range(n1 + n2))
    w_ref = ref.get_weights()
    _, step_ref, scale_ref = ref.state()
    path = tmp_path / "ckpt.rfdmlp"
    ref.set_weights(w0)
    run(ref, range(n1))
    ref.save(path)
    ref.set_weights(omd.init_weights(len(REFS), seed=99))           # the state is gone from ref
    fresh = rfd.Mlp(env["ctx"], env["g"], env["psd"], REFS)
    fresh.load(path)
    run(fresh, range(n1, n1 + n2))
    w_res = fresh.get_weights()
    _, step_res, scale_res = fresh.state()
    assert step_res == step_ref == n1 + n2
    assert scale_res == scale_ref
    assert np.array_equal(w_res.view(np.uint32), w_ref.view(np.uint32))
    # inference from the loaded network equals the original's on the same inputs
    P, ro = dense["held"].params()[:64], dense["held"].ref_of_tmpl[:64]
    outs = []
    for net in (fresh, ref):
        if net is ref:
            ref.load(path)
            run(ref, range(n1, n1 + n2))
        taps = torch.zeros((len(P), K), dtype=torch.complex64, device="cuda")
        lag = torch.zeros(len(P), dtype=torch.int32, device="cuda")
        sig = torch.zeros(len(P), dtype=torch.float64, device="cuda")
        net.infer(P, ro, taps, lag, sig)
        outs.append(taps.cpu().numpy())
    assert np.array_equal(outs[0].view(np.uint32), outs[1].view(np.uint32))
    # a network object for other references refuses the checkpoint
    other = rfd.Mlp(env["ctx"], env["g"], env["psd"], REFS[::-1].copy())
    with pytest.raises(rfd.RfdError) as ei:
        other.load(path)
    assert ei.value.status == _native.RFD_ERR_ARG
    other.close()
    fresh.close()

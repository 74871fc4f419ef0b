"""Chi^2-fitted ridge taps (Sec. V.A) on the GPU against the oracle (oracle/fit.py).

* fixed K: lags identical, taps (Levinson, FP64, stored FP32) equal to the oracle's dense solve,
  sigma_eff and the closed-form match equal;
* dynamic K: every template gets the oracle's bucket (the smallest whose fitted match reaches
  the target) unless its match at the deciding bucket lies within 1e-7 of the target;
* the whole path with fitted taps (tensor cores) gives the oracle's triggers.
"""
import numpy as np
import pytest

import workload
from oracle import fit
from tests.oracle_pipeline import OracleRun

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402
from tests.gpu_pipeline import GpuRun  # noqa: E402
from tests.test_gpu_parity import EPS, TOL_TC, amb_cap, compare_triggers, n_oracle, snr_errors  # noqa: E402

RIDGE = 1e-6


@pytest.fixture(scope="module")
def c1():
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg)
    gpu = GpuRun(cfg, bank, data)
    return cfg, bank, data, gpu


def _fit_gpu(gpu, bank, idx, K=None, buckets=None, target=0.99, k_stride=128):
    J = len(idx)
    taps = torch.zeros((J, k_stride), dtype=torch.complex64, device="cuda")
    lag = torch.zeros(J, dtype=torch.int32, device="cuda")
    sig = torch.zeros(J, dtype=torch.float64, device="cuda")
    mat = torch.zeros(J, dtype=torch.float64, device="cuda")
    kout = torch.zeros(J, dtype=torch.int32, device="cuda")
    rfd.make_taps_fit(gpu.ctx, gpu.grid, gpu.psd, bank.ref_params(), bank.params()[idx], bank.ref_of_tmpl[idx],
                      None if K is None else np.full(J, K, dtype=np.int32), k_stride, 0.1, taps, lag, sig, mat,
                      ridge=RIDGE, buckets=buckets, match_target=target, k_out=kout)
    torch.cuda.synchronize()
    return (taps.cpu().numpy(), lag.cpu().numpy(), sig.cpu().numpy(), mat.cpu().numpy(), kout.cpu().numpy(),
            taps, lag, sig)


def test_fitted_taps_match_oracle(c1):
    cfg, bank, data, gpu = c1
    idx = np.arange(12)
    K = 64
    taps, lag, sig, mat, _, *_ = _fit_gpu(gpu, bank, idx, K=K)
    for i, j in enumerate(idx):
        o = fit.design(cfg.fs, cfg.n, cfg.f_low, bank.params()[j], bank.ref_params()[bank.ref_of_tmpl[j]],
                       data.psd, K, RIDGE, cfg.tukey_alpha, cfg.pn_flags)
        assert lag[i] == o["lag"], (j, lag[i], o["lag"])
        err = np.linalg.norm(taps[i, :K] - o["taps"]) / np.linalg.norm(o["taps"])
        assert err < 1e-6, (j, err)
        assert np.all(taps[i, K:] == 0)
        assert abs(sig[i] / o["sigma_eff"] - 1) < 1e-8, j
        assert abs(mat[i] - o["match"]) < 1e-8, (j, mat[i], o["match"])


def test_dynamic_k_matches_oracle(c1):
    cfg, bank, data, gpu = c1
    idx = np.arange(10)
    buckets, target = [16, 32, 64, 128], 0.99
    taps, lag, sig, mat, kk, *_ = _fit_gpu(gpu, bank, idx, buckets=buckets, target=target)
    for i, j in enumerate(idx):
        o = fit.design_dynamic(cfg.fs, cfg.n, cfg.f_low, bank.params()[j], bank.ref_params()[bank.ref_of_tmpl[j]],
                               data.psd, buckets, target, RIDGE, cfg.tukey_alpha, cfg.pn_flags)
        if abs(o["match"] - target) < 1e-7:
            continue
        assert kk[i] == o["K"], (j, kk[i], o["K"])
        assert abs(mat[i] - o["match"]) < 1e-8
        assert lag[i] == o["lag"]


def test_fitted_taps_filter_to_oracle_triggers(c1):
    cfg, bank, data, gpu = c1
    ora = OracleRun(cfg, bank, data)
    idx = np.arange(bank.n_tmpl)
    K = cfg.k
    _, _, _, _, _, taps, lag, sig = _fit_gpu(gpu, bank, idx, K=K, k_stride=K)
    t = {"taps": taps, "lag": lag, "sigma": sig, "K": np.full(len(idx), K, np.int32), "k_stride": K, "idx": idx}
    halo = K - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP16X3)
    trig, _ = gpu.ratio_filter(t, q, e, rfd.PREC_FP16X3, halo)
    sets = {}
    for j in idx:
        o = fit.design(cfg.fs, cfg.n, cfg.f_low, bank.params()[j], bank.ref_params()[bank.ref_of_tmpl[j]],
                       data.psd, K, RIDGE, cfg.tukey_alpha, cfg.pn_flags)
        sets[j] = ora.triggers(ora.snr(j, {"taps": o["taps"], "lag": o["lag"], "sigma_eff": o["sigma_eff"]}),
                               EPS[rfd.PREC_FP16X3])
    assert compare_triggers(trig, sets, TOL_TC, idx, cfg.window) <= amb_cap(n_oracle(sets, idx))
    assert snr_errors(trig, sets, idx) < EPS[rfd.PREC_FP16X3]

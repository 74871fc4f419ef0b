"""Sub-band chi^2 through the ratio filter on the GPU against the oracle (oracle/chisq.py).

* band edges identical (integer decisions from the same FP64 running sum);
* sub-band reference series within 1e-5 of their rms (FP32 Stockham against the FP64 oracle),
  and adding up to the full-band reference series;
* each template's band shares u_b within 1e-5;
* at every trigger of the C1 bank: chi^2 within 1e-3 relative (plus 1e-3 of the degrees of
  freedom) of the oracle's, and the sub-band SNRs add up to the trigger's z.
"""
import numpy as np
import pytest

import workload
from oracle import chisq, waveform as wf
from tests.oracle_pipeline import OracleRun

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402
from tests.gpu_pipeline import GpuRun  # noqa: E402

P = 8


@pytest.fixture(scope="module")
def setup():
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg)
    gpu = GpuRun(cfg, bank, data)
    sb = rfd.Subband(gpu.ctx, gpu.grid, gpu.psd, bank.ref_params(), P)
    yield cfg, bank, data, gpu, sb
    sb.close()


def test_edges_and_band_series(setup):
    cfg, bank, data, gpu, sb = setup
    df = cfg.fs / cfg.n
    h_ref = wf.template(cfg.fs, cfg.n, cfg.f_low, bank.ref_params()[0])
    e_ora = chisq.band_edges(h_ref, data.psd, df, P)
    e_gpu = sb.edges()[0]
    assert np.array_equal(e_gpu, e_ora), (e_gpu, e_ora)
    href = gpu.templates(bank.ref_params())
    halo = cfg.k - 1
    qb = sb.filter_reference(gpu.d, gpu.psd, href, halo).cpu().numpy()
    ora = chisq.band_series(data.dtilde.astype(np.complex64).astype(np.complex128), h_ref, data.psd, df, cfg.n, e_ora)
    for b in range(P):
        rms = np.sqrt(np.mean(np.abs(ora[b]) ** 2))
        assert np.max(np.abs(qb[0, b, : cfg.n] - ora[b])) <= 1e-5 * rms, b
        assert np.array_equal(qb[0, b, cfg.n: cfg.n + halo], qb[0, b, :halo])     # wrap halo
    q_full, _, ld = gpu.filter_reference(halo, rfd.PREC_FP32)
    q_full = q_full.view(torch.complex64).cpu().numpy()[: cfg.n]
    assert np.max(np.abs(qb[0, :, : cfg.n].sum(axis=0) - q_full)) <= 1e-5 * np.sqrt(np.mean(np.abs(q_full) ** 2))


def test_shares_and_chi2_at_triggers(setup):
    cfg, bank, data, gpu, sb = setup
    df = cfg.fs / cfg.n
    ora = OracleRun(cfg, bank, data)
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP32)
    # a lower threshold than the search's gives a few hundred triggers to check
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], rfd.PREC_FP32, cfg.window, 12.0, halo)
    plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
    cand = torch.zeros((1 << 20) * 24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan.ratio_filter_batch(q, e, cand, cnt)
    tb = torch.zeros((1 << 16) * 20, dtype=torch.uint8, device="cuda")
    nt = rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, tb)
    plan.close()
    trig = rfd.triggers_to_numpy(tb, nt)
    assert nt > 100
    href = gpu.templates(bank.ref_params())
    qb = sb.filter_reference(gpu.d, gpu.psd, href, halo)
    kd = torch.from_numpy(t["K"].astype(np.int32)).cuda()
    u = sb.shares(gpu.psd, t["taps"], kd, t["lag"], bank.ref_of_tmpl)
    chi2, zb = sb.chi2(qb, halo, t["taps"], kd, t["lag"], t["sigma"], u, bank.ref_of_tmpl, tb, nt, zb=True)
    chi2, zb, u = chi2.cpu().numpy(), zb.cpu().numpy(), u.cpu().numpy()
    h_ref = wf.template(cfg.fs, cfg.n, cfg.f_low, bank.ref_params()[0])
    edges = chisq.band_edges(h_ref, data.psd, df, P)
    qb_ora = chisq.band_series(ora.d, h_ref, data.psd, df, cfg.n, edges)
    Cb = chisq.band_autocorr(h_ref, data.psd, df, cfg.n, edges, cfg.k - 1)
    dof = 2 * (P - 1)
    checked = 0
    for j in sorted(set(trig["j"].tolist())):
        o = ora.design(int(j), cfg.k, with_match=False)
        rows = np.nonzero(trig["j"] == j)[0]
        c_ora, zb_ora, u_ora = chisq.subband_chi2(qb_ora, o["taps"], o["lag"], o["sigma_eff"], Cb,
                                                  trig["t"][rows].astype(np.int64))
        assert np.max(np.abs(u[j] - u_ora)) <= 1e-5, j
        for i, r in enumerate(rows):
            assert abs(chi2[r] - c_ora[i]) <= 1e-3 * c_ora[i] + 1e-3 * dof, (j, chi2[r], c_ora[i])
            z = complex(trig["zr"][r], trig["zi"][r])
            assert abs(zb[r].sum() - z) <= 1e-4 * abs(z)
            checked += 1
    assert checked == nt

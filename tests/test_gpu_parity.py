"""GPU parity: every C-ABI step against the FP64 oracle on the same seeded inputs.

Tolerances.  The method's targets: SNR |z| within 1e-3 relative on the tensor-core path and
1e-5 on the FP32 path (TOL_TC, TOL_FP32).  Each arithmetic path also has a much tighter error
bound EPS[precision] (relative |z| error at trigger samples; the full-series tests below
measure the largest error over every sample of every template, relative to rms |z|, and the
bounds sit about 2x above those measurements).  Every parity test asserts its triggers' |z|
within EPS, and trigger (j, w, t) bit-exact except in windows the oracle flags ambiguous under
EPS (a peak within 4 EPS of the threshold, or a runner-up within 4 EPS of the peak: the only
windows an error within EPS can decide differently); at most 1 % of the oracle's trigger
windows may be skipped that way.  Lags bit-exact; sigma_eff and match within 1e-9 (FP64 on
both sides); taps within the complex64 rounding of their FP64 values.
"""
import math

import numpy as np
import pytest

import workload
from tests.oracle_pipeline import OracleRun

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402
from tests.gpu_pipeline import GpuRun  # noqa: E402

TOL_FP32 = 1e-5
TOL_TC = 1e-3
# error bounds of the arithmetic paths (relative |z| error), per plan precision
EPS = {rfd.PREC_FP32: 2e-6, rfd.PREC_FP16X3: 2e-5, rfd.PREC_BF16X3: 2e-4}
# full-series bounds: max |z_gpu - z_oracle| over a template's series / rms |z_oracle|.  Measured
# on GB300 over C1 and the ragged bank (the largest over the kernels of each precision): FP32
# 3.2e-6 (direct FIR) / 2.6e-6 (block FFT); FP16x3 5.3e-6; BF16x3 1.8e-4 (its hi + lo split keeps
# about 16 significant bits, so it is the precision whose band is widest)
EPS_SERIES = {rfd.PREC_FP32: 8e-6, rfd.PREC_FP16X3: 1.2e-5, rfd.PREC_BF16X3: 4e-4}


def amb_cap(n_or):
    """Ambiguous windows allowed: 1 % of the oracle's trigger windows, rounded up."""
    return int(math.ceil(0.01 * n_or))


@pytest.fixture(scope="module")
def ctx():
    from paper_2601_18835_gb300 import build
    build.build()
    c = rfd.Context(0)
    yield c
    c.close()


def compare_triggers(gpu_trig, oracle_sets, tol, js, W):
    """gpu_trig: structured array (j, t, snr2, zr, zi); oracle_sets: {j: (triggers, ambiguous)}
    with the ambiguity flags taken under the path's error bound.  Every non-ambiguous window
    must agree in (j, w, t) and in |z| within tol.  Returns the number of ambiguous windows
    skipped."""
    n_amb = 0
    for j in js:
        ot, amb = oracle_sets[j]
        amb = set(amb)
        o_by_w = {x["w"]: x for x in ot}
        g_by_w = {}
        for r in gpu_trig[gpu_trig["j"] == j]:
            t = int(r["t"])
            assert t // W not in g_by_w, ("two gpu triggers in one window", j, t)
            g_by_w[t // W] = (t, float(r["snr2"]), complex(float(r["zr"]), float(r["zi"])))
        for w in sorted(set(o_by_w) | set(g_by_w)):
            if w in amb:
                n_amb += 1
                continue
            assert w in o_by_w, ("gpu-only trigger", j, w, g_by_w.get(w))
            assert w in g_by_w, ("oracle-only trigger", j, w, o_by_w[w])
            t, p, z = g_by_w[w]
            assert t == o_by_w[w]["t"], (j, w, t, o_by_w[w]["t"])
            za = abs(o_by_w[w]["z"])
            assert abs(math.sqrt(p) - za) <= tol * za, (j, w, math.sqrt(p), za)
            assert abs(z - o_by_w[w]["z"]) <= 4 * tol * za
    return n_amb


# --------------------------------------------------------------------------- FFT
@pytest.mark.parametrize("n,batch", [(1024, 3), (8192, 2), (16384, 2), (32768, 1), (524288, 2), (1048576, 1)])
def test_ifft_matches_numpy(ctx, n, batch):
    rng = np.random.default_rng(n)
    x = (rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    rfd.ifft_c2c(ctx, xd, out)
    ref = np.fft.ifft(x.astype(np.complex128), axis=1) * n
    got = out.cpu().numpy()
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert np.max(np.abs(got - ref)) / rms < 2e-6


# every size class of the transform: one pass per radix below 2^12, the two-pass (four-step)
# form from 2^12 (N1 = N2 = 64) to 2^22 (N1 = 2048, N2 = 2048: the largest shared-memory tile),
# odd log2 n (N1 = 2 N2) and one pass per radix again above 2^22
@pytest.mark.parametrize("n,batch", [(256, 5), (2048, 3), (4096, 3), (8192, 2), (131072, 2), (524288, 3),
                                     (4194304, 1), (8388608, 1)])
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft_both_directions_and_precisions(ctx, n, batch, fp64, inverse):
    rng = np.random.default_rng(n + 7 * batch)
    x = rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n))
    x = x.astype(np.complex128 if fp64 else np.complex64)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    rfd.fft_c2c(ctx, xd, out, inverse)
    ref = np.fft.ifft(x.astype(np.complex128), axis=1) * n if inverse else np.fft.fft(x.astype(np.complex128), axis=1)
    got = out.cpu().numpy()
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    # radix-16 Stockham error grows like log2 n eps: 2e-6 (FP32) and 1e-14 (FP64) of the rms
    assert np.max(np.abs(got - ref)) / rms < (1e-14 if fp64 else 2e-6)


# --------------------------------------------------------------------------- templates
def test_gen_templates_match_oracle(ctx):
    from oracle import waveform as wf
    cfg = workload.get_config(1)
    bank = workload.make_bank(cfg)
    p = bank.params()[:8]
    g = rfd.grid(cfg.fs, cfg.n, cfg.f_low)
    h = torch.zeros((8, cfg.n // 2 + 1), dtype=torch.complex64, device="cuda")
    rfd.gen_templates(ctx, g, p, h)
    got = h.cpu().numpy()
    for i in range(8):
        ref = wf.template(cfg.fs, cfg.n, cfg.f_low, p[i])
        assert np.array_equal(np.nonzero(got[i])[0], np.nonzero(ref)[0])
        assert np.max(np.abs(got[i] - ref)) <= 1e-6 * np.max(np.abs(ref))


# --------------------------------------------------------------------------- C1 end to end
@pytest.fixture(scope="module")
def c1(ctx):
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg)
    return cfg, bank, data, OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)


def test_filter_reference_fp32_and_split(c1):
    cfg, bank, data, ora, gpu = c1
    halo = cfg.k - 1
    q, e, ld = gpu.filter_reference(halo, rfd.PREC_FP32)
    qg = q.view(torch.complex64).cpu().numpy()[:ld]
    qo = ora.q_ref(0)
    rms = np.sqrt(np.mean(np.abs(qo) ** 2))
    assert np.max(np.abs(qg[:cfg.n] - qo)) / rms < TOL_FP32
    assert np.array_equal(qg[cfg.n:cfg.n + halo], qg[:halo])
    assert int(e.item()) == 0
    for prec, ht, tol in ((rfd.PREC_FP16X3, torch.float16, 2e-6), (rfd.PREC_BF16X3, torch.bfloat16, 2e-4)):
        qs, es, _ = gpu.filter_reference(halo, prec)
        planes = qs.view(ht).float().cpu().numpy().astype(np.float64).reshape(4, ld)
        scale = 2.0 ** (-int(es.item()))
        rec = ((planes[0] + planes[2]) + 1j * (planes[1] + planes[3])) * scale
        assert np.max(np.abs(rec[:cfg.n] - qo)) / rms < tol
        assert np.array_equal(planes[:, cfg.n:cfg.n + halo], planes[:, :halo])
        assert np.all(planes[:, cfg.n + halo:] == 0)


def test_make_taps_c1_matches_oracle(c1):
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k)
    taps = t["taps"].cpu().numpy()
    lag = t["lag"].cpu().numpy()
    sig = t["sigma"].cpu().numpy()
    mat = t["match"].cpu().numpy()
    for j in range(bank.n_tmpl):
        o = ora.design(j, cfg.k)
        assert lag[j] == o["lag"], (j, lag[j], o["lag"])
        assert np.max(np.abs(taps[j] - o["taps"])) <= 2e-7 * max(1e-30, np.max(np.abs(o["taps"]))) + 1e-12
        assert abs(sig[j] / o["sigma_eff"] - 1) < 1e-9
        assert abs(mat[j] - o["match"]) < 1e-9
    # identity slot: delta taps at K/2
    assert lag[0] == -cfg.k // 2
    d = np.zeros(cfg.k, complex)
    d[cfg.k // 2] = 1
    assert np.max(np.abs(taps[0] - d)) < 1e-7


def test_c1_triggers_fp32(c1):
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP32)
    trig, ncand = gpu.ratio_filter(t, q, e, rfd.PREC_FP32, halo)
    sets = {}
    for j in range(bank.n_tmpl):
        o = ora.design(j, cfg.k, with_match=False)
        sets[j] = ora.triggers(ora.snr(j, o), EPS[rfd.PREC_FP32])
    n_amb = compare_triggers(trig, sets, TOL_FP32, range(bank.n_tmpl), cfg.window)
    assert n_amb <= amb_cap(n_oracle(sets, range(bank.n_tmpl)))
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[rfd.PREC_FP32]
    # the injected template fires at the injected sample
    m0, snr, phi, slot = data.injections[0]
    hit = trig[(trig["j"] == slot)]
    assert len(hit) >= 1 and abs(int(hit["t"][np.argmax(hit["snr2"])]) - m0) <= 1


def test_c1_findchirp_matches_oracle(c1):
    cfg, bank, data, ora, gpu = c1
    cap = 1 << 18
    cand = torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    rfd.findchirp(gpu.ctx, gpu.grid, gpu.d, gpu.psd, gpu.templates(bank.params()), cfg.window, cfg.threshold,
                  cand, cnt)
    trig = torch.zeros(cap * 20, dtype=torch.uint8, device="cuda")
    nt = rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, trig)
    tr = rfd.triggers_to_numpy(trig, nt)
    sets = {j: ora.triggers(ora.findchirp(j), EPS[rfd.PREC_FP32]) for j in range(bank.n_tmpl)}
    assert compare_triggers(tr, sets, TOL_FP32, range(bank.n_tmpl), cfg.window) <= amb_cap(
        n_oracle(sets, range(bank.n_tmpl)))
    assert snr_errors(tr, sets, range(bank.n_tmpl)) < EPS[rfd.PREC_FP32]


def test_ratio_peak_within_one_percent_of_findchirp_gpu(c1):
    cfg, bank, data, ora, gpu = c1
    m0, snr, phi, slot = data.injections[0]
    t = gpu.make_taps(cfg.k, match=True)
    assert t["match"].cpu().numpy()[slot] >= 0.99
    q, e, _ = gpu.filter_reference(cfg.k - 1, rfd.PREC_FP32)
    trig, _ = gpu.ratio_filter(t, q, e, rfd.PREC_FP32, cfg.k - 1)
    pr = float(trig[trig["j"] == slot]["snr2"].max())
    cap = 1 << 16
    cand = torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    rfd.findchirp(gpu.ctx, gpu.grid, gpu.d, gpu.psd, gpu.templates(bank.params()[slot:slot + 1]), cfg.window,
                  cfg.threshold, cand, cnt)
    tb = torch.zeros(cap * 20, dtype=torch.uint8, device="cuda")
    nt = rfd.find_triggers(gpu.ctx, 1, cand, cnt, tb)
    pf = float(rfd.triggers_to_numpy(tb, nt)["snr2"].max())
    assert abs(math.sqrt(pr / pf) - 1) < 0.01


# --------------------------------------------------------------------------- edge cases
def test_ragged_bank_uneven_taps_and_window(ctx):
    """37 templates (not a multiple of the tile), per-template K from 2 to 96, a window that
    does not divide n, and a low threshold so that many windows fire."""
    cfg = workload.small_config(1, n_tmpl=37, window=37, threshold=6.0)
    bank, data = workload.make_workload(cfg)
    rng = np.random.default_rng(7)
    K = (2 * rng.integers(1, 49, size=bank.n_tmpl)).astype(np.int32)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=128, match=False)
    halo = int(K.max()) - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP32)
    trig, ncand = gpu.ratio_filter(t, q, e, rfd.PREC_FP32, halo, cand_cap=1 << 22)
    lag = t["lag"].cpu().numpy()
    sets = {}
    for j in range(bank.n_tmpl):
        o = ora.design(j, int(K[j]), with_match=False)
        assert lag[j] == o["lag"]
        sets[j] = ora.triggers(ora.snr(j, o), EPS[rfd.PREC_FP32])
    n_or = n_oracle(sets, range(bank.n_tmpl))
    assert n_or > 1000
    n_amb = compare_triggers(trig, sets, TOL_FP32, range(bank.n_tmpl), cfg.window)
    assert n_amb <= amb_cap(n_or)
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[rfd.PREC_FP32]


def test_candidate_overflow_is_reported(c1):
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    q, e, _ = gpu.filter_reference(cfg.k - 1, rfd.PREC_FP32)
    with pytest.raises(rfd.RfdError) as ei:
        gpu.ratio_filter(t, q, e, rfd.PREC_FP32, cfg.k - 1, cand_cap=2)
    assert ei.value.status == -7 and ei.value.needed > 2


def test_bad_arguments_are_rejected(ctx):
    g = rfd.grid(1024.0, 1000, 30.0)                      # not a power of two
    h = torch.zeros((1, 501), dtype=torch.complex64, device="cuda")
    with pytest.raises(rfd.RfdError) as ei:
        rfd.gen_templates(ctx, g, np.array([[1.4, 1.4, 0, 0, 0]]), h)
    assert ei.value.status == -2
    g = rfd.grid(1024.0, 16384, 30.0)
    with pytest.raises(rfd.RfdError) as ei:
        rfd.gen_templates(ctx, g, np.array([[-1.0, 1.4, 0, 0, 0]]), torch.zeros((1, 8193), dtype=torch.complex64,
                                                                              device="cuda"))
    assert ei.value.status == -1


# --------------------------------------------------------------------------- full size, sampled
@pytest.mark.slow
def test_c2_full_size_fp32_sampled(ctx):
    """The 256 s / 2048 Hz bank (4096 templates, 16 references, K = 128) end to end on the GPU;
    the oracle checks a stratified sample: every injected template plus one per reference."""
    cfg = workload.get_config(2)
    bank, data = workload.make_workload(cfg)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(cfg.k, match=True)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP32)
    trig, ncand = gpu.ratio_filter(t, q, e, rfd.PREC_FP32, halo)
    lag, sig, mat = (t[k].cpu().numpy() for k in ("lag", "sigma", "match"))
    sample = sorted({s for (_, _, _, s) in data.injections}
                    | {int(np.nonzero(bank.ref_of_tmpl == r)[0][0]) for r in range(0, bank.n_ref, 4)})
    sets = {}
    for j in sample:
        o = ora.design(j, cfg.k)
        assert lag[j] == o["lag"]
        assert abs(sig[j] / o["sigma_eff"] - 1) < 1e-9
        assert abs(mat[j] - o["match"]) < 1e-8
        z = ora.snr(j, o)
        sets[j] = ora.triggers(z, EPS[rfd.PREC_FP32])
        g = trig[trig["j"] == j]
        if len(g):
            zo = ora.snr_at(j, o, g["t"].astype(np.int64))
            assert np.max(np.abs(np.sqrt(g["snr2"]) - np.abs(zo)) / np.abs(zo)) < EPS[rfd.PREC_FP32]
    assert compare_triggers(trig, sets, TOL_FP32, sample, cfg.window) <= amb_cap(n_oracle(sets, sample))


# --------------------------------------------------------------------------- tensor-core path
TC_PRECISIONS = [("fp16x3", 1), ("bf16x3", 2)]
# the two tensor-core kernels: time on M with templates on N (K <= 64 by default), and
# templates on M with time on N (the long-tap kernel, K > 64 by default), each forced for all;
# and the block-FFT kernel (FP32 transforms of the split series' reconstruction) for all
TC_KERNELS = [("time_on_m", {"long_k": 512}), ("templates_on_m", {"long_k": 0}), ("block_fft", {"fft_k": 0})]


def snr_errors(trig, sets, js):
    """Largest relative error over the GPU triggers that the oracle also has (same t): of |z|,
    and of the complex z."""
    worst = 0.0
    for j in js:
        o_by_t = {x["t"]: x for x in sets[j][0]}
        for r in trig[trig["j"] == j]:
            x = o_by_t.get(int(r["t"]))
            if x is not None:
                za = abs(x["z"])
                zg = complex(float(r["zr"]), float(r["zi"]))
                worst = max(worst, abs(math.sqrt(float(r["snr2"])) / za - 1.0), 0.5 * abs(zg - x["z"]) / za)
    return worst


def n_oracle(sets, js):
    return sum(len(sets[j][0]) for j in js)


@pytest.mark.parametrize("kernel,opts", TC_KERNELS)
@pytest.mark.parametrize("name,prec", TC_PRECISIONS)
def test_c1_triggers_tensor_core(c1, name, prec, kernel, opts):
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, prec)
    trig, ncand = gpu.ratio_filter(t, q, e, prec, halo, options=opts)
    sets = {}
    for j in range(bank.n_tmpl):
        o = ora.design(j, cfg.k, with_match=False)
        sets[j] = ora.triggers(ora.snr(j, o), EPS[prec])
    n_amb = compare_triggers(trig, sets, TOL_TC, range(bank.n_tmpl), cfg.window)
    assert n_amb <= amb_cap(n_oracle(sets, range(bank.n_tmpl)))
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[prec]


@pytest.mark.parametrize("kernel,opts", TC_KERNELS)
@pytest.mark.parametrize("name,prec", TC_PRECISIONS)
def test_ragged_bank_tensor_core(ctx, name, prec, kernel, opts):
    """37 templates, K from 2 to 96 (tiles padded to 16-tap steps), window 37, low threshold."""
    cfg = workload.small_config(1, n_tmpl=37, window=37, threshold=6.0)
    bank, data = workload.make_workload(cfg)
    rng = np.random.default_rng(7)
    K = (2 * rng.integers(1, 49, size=bank.n_tmpl)).astype(np.int32)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=128, match=False)
    halo = int(((K.max() + 15) // 16) * 16) - 1
    q, e, _ = gpu.filter_reference(halo, prec)
    trig, ncand = gpu.ratio_filter(t, q, e, prec, halo, cand_cap=1 << 22, options=opts)
    sets = {}
    for j in range(bank.n_tmpl):
        o = ora.design(j, int(K[j]), with_match=False)
        sets[j] = ora.triggers(ora.snr(j, o), EPS[prec])
    n_or = n_oracle(sets, range(bank.n_tmpl))
    assert n_or > 1000
    assert compare_triggers(trig, sets, TOL_TC, range(bank.n_tmpl), cfg.window) <= amb_cap(n_or)
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[prec]


@pytest.mark.parametrize("name,prec", TC_PRECISIONS[:1])
def test_long_taps_tensor_core(ctx, name, prec):
    """K = 320 and 512 (tiles of 32 templates, 20 and 32 MMA steps) next to K = 64 (64 per tile)."""
    cfg = workload.small_config(1, n_tmpl=80, threshold=9.0)
    bank, data = workload.make_workload(cfg)
    K = np.where(np.arange(bank.n_tmpl) % 3 == 0, 320, np.where(np.arange(bank.n_tmpl) % 3 == 1, 512, 64))
    K = K.astype(np.int32)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=512, match=False)
    halo = 511
    q, e, _ = gpu.filter_reference(halo, prec)
    trig, ncand = gpu.ratio_filter(t, q, e, prec, halo, cand_cap=1 << 22)
    js = list(range(0, bank.n_tmpl, 5))
    sets = {}
    for j in js:
        o = ora.design(j, int(K[j]), with_match=False)
        sets[j] = ora.triggers(ora.snr(j, o), EPS[prec])
    n_or = n_oracle(sets, js)
    assert n_or > 100
    assert compare_triggers(trig, sets, TOL_TC, js, cfg.window) <= amb_cap(n_or)
    assert snr_errors(trig, sets, js) < EPS[prec]


def test_block_fft_fp32_c1_and_ragged(ctx, c1):
    """The block-FFT kernel on an FP32 plan: C1 (K = 64) and a ragged bank (K from 2 to 96,
    window 37, threshold 6; the last 2048-sample block only partly valid), FP32 tolerance."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP32)
    trig, _ = gpu.ratio_filter(t, q, e, rfd.PREC_FP32, halo, options={"fft_k": 0})
    sets = {j: ora.triggers(ora.snr(j, ora.design(j, cfg.k, with_match=False)), EPS[rfd.PREC_FP32])
            for j in range(bank.n_tmpl)}
    assert compare_triggers(trig, sets, TOL_FP32, range(bank.n_tmpl), cfg.window) <= amb_cap(
        n_oracle(sets, range(bank.n_tmpl)))
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[rfd.PREC_FP32]
    cfg = workload.small_config(1, n_tmpl=37, window=37, threshold=6.0)
    bank, data = workload.make_workload(cfg)
    rng = np.random.default_rng(7)
    K = (2 * rng.integers(1, 49, size=bank.n_tmpl)).astype(np.int32)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=128, match=False)
    halo = int(K.max()) - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP32)
    trig, _ = gpu.ratio_filter(t, q, e, rfd.PREC_FP32, halo, cand_cap=1 << 22, options={"fft_k": 0})
    sets = {j: ora.triggers(ora.snr(j, ora.design(j, int(K[j]), with_match=False)), EPS[rfd.PREC_FP32])
            for j in range(bank.n_tmpl)}
    n_or = n_oracle(sets, range(bank.n_tmpl))
    assert n_or > 1000
    assert compare_triggers(trig, sets, TOL_FP32, range(bank.n_tmpl), cfg.window) <= amb_cap(n_or)
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[rfd.PREC_FP32]


def test_block_fft_next_to_tensor_cores(ctx):
    """K = 64 on the tensor cores and K = 320 / 512 on the block-FFT kernel (fft_k = 256) in one
    plan and one call: every sampled template matches the oracle."""
    cfg = workload.small_config(1, n_tmpl=80, threshold=9.0)
    bank, data = workload.make_workload(cfg)
    K = np.where(np.arange(bank.n_tmpl) % 3 == 0, 320, np.where(np.arange(bank.n_tmpl) % 3 == 1, 512, 64))
    K = K.astype(np.int32)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=512, match=False)
    halo = 511
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP16X3)
    trig, _ = gpu.ratio_filter(t, q, e, rfd.PREC_FP16X3, halo, cand_cap=1 << 22, options={"fft_k": 256})
    js = list(range(0, bank.n_tmpl, 4))
    sets = {j: ora.triggers(ora.snr(j, ora.design(j, int(K[j]), with_match=False)), EPS[rfd.PREC_FP16X3])
            for j in js}
    n_or = n_oracle(sets, js)
    assert n_or > 100
    assert compare_triggers(trig, sets, TOL_TC, js, cfg.window) <= amb_cap(n_or)
    assert snr_errors(trig, sets, js) < EPS[rfd.PREC_FP16X3]


@pytest.mark.parametrize("name,prec", TC_PRECISIONS)
def test_last_partial_tile_on_block_fft(ctx, name, prec):
    """fft_rem: 75 templates of one reference fill one 64-template tile of the long-tap kernel
    and leave 11, which go to the block-FFT kernel (fft_rem = 16) instead of a padded tile; both
    parts of the call match the oracle, and the plan keeps every template exactly once."""
    cfg = workload.small_config(1, n_tmpl=75, threshold=9.0)
    bank, data = workload.make_workload(cfg)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, prec)
    trig, _ = gpu.ratio_filter(t, q, e, prec, halo, options={"long_k": 0, "fft_rem": 16})
    sets = {j: ora.triggers(ora.snr(j, ora.design(j, cfg.k, with_match=False)), EPS[prec])
            for j in range(bank.n_tmpl)}
    n_or = n_oracle(sets, range(bank.n_tmpl))
    assert n_or > 20
    assert compare_triggers(trig, sets, TOL_TC, range(bank.n_tmpl), cfg.window) <= amb_cap(n_or)
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[prec]
    # the last 11 templates of the (stable, equal-K) order, 64..74, ran on the block-FFT kernel:
    # their values (FP32 transforms) differ from the tensor cores' in the last bits; every other
    # template's triggers are bit-identical to the plan without fft_rem
    trig_tc, _ = gpu.ratio_filter(t, q, e, prec, halo, options={"long_k": 0})
    a = {(int(x["j"]), int(x["t"]) // cfg.window): x for x in trig}
    b = {(int(x["j"]), int(x["t"]) // cfg.window): x for x in trig_tc}
    diff_j = {key[0] for key in set(a) | set(b) if key not in a or key not in b or a[key].tobytes() != b[key].tobytes()}
    assert diff_j and diff_j <= set(range(64, 75))
    # the plan reports the same assignment
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], prec, cfg.window, cfg.threshold, halo,
                    options={"long_k": 0, "fft_rem": 16})
    kern = plan.template_kernels()
    plan.close()
    assert np.array_equal(kern, np.where(np.arange(bank.n_tmpl) >= 64, 3, 2))


@pytest.mark.slow
@pytest.mark.parametrize("name,prec", TC_PRECISIONS)
def test_c2_full_size_tensor_core_sampled(ctx, name, prec):
    """The 4096-template, 2^19-sample bank on the tensor-core path; oracle on a stratified sample;
    every GPU trigger of a sampled template is re-evaluated by the oracle at its sample."""
    cfg = workload.get_config(2)
    bank, data = workload.make_workload(cfg)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, prec)
    trig, ncand = gpu.ratio_filter(t, q, e, prec, halo)
    sample = sorted({s for (_, _, _, s) in data.injections}
                    | {int(np.nonzero(bank.ref_of_tmpl == r)[0][-1]) for r in range(0, bank.n_ref, 3)})
    sets = {}
    for j in sample:
        o = ora.design(j, cfg.k, with_match=False)
        sets[j] = ora.triggers(ora.snr(j, o), EPS[prec])
        g = trig[trig["j"] == j]
        if len(g):
            zo = ora.snr_at(j, o, g["t"].astype(np.int64))
            assert np.max(np.abs(np.sqrt(g["snr2"]) - np.abs(zo)) / np.abs(zo)) < EPS[prec]
    assert compare_triggers(trig, sets, TOL_TC, sample, cfg.window) <= amb_cap(n_oracle(sets, sample))


@pytest.mark.slow
def test_c5_grid_long_taps_sampled(ctx):
    """The C5 grid (512 s at 2048 Hz, n = 2^20, f_low 45 Hz, subsolar masses) with K = 512 on
    the templates-on-M kernel: 256 templates over 2 references, every GPU trigger of a sampled
    template re-evaluated by the oracle at its sample, and the sampled templates' oracle
    trigger sets matched window by window."""
    cfg = workload.small_config(5, n_tmpl=256, n_ref=2)
    bank, data = workload.make_workload(cfg)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP16X3)
    trig, ncand = gpu.ratio_filter(t, q, e, rfd.PREC_FP16X3, halo, cand_cap=1 << 22)
    inj = sorted({s for (_, _, _, s) in data.injections})
    sample = sorted(set(inj[:2]) | {int(np.nonzero(bank.ref_of_tmpl == r)[0][-1]) for r in range(bank.n_ref)})
    sets = {}
    checked = 0
    for j in sample:
        o = ora.design(j, cfg.k, with_match=False)
        sets[j] = ora.triggers(ora.snr(j, o), EPS[rfd.PREC_FP16X3])
        g = trig[trig["j"] == j]
        if len(g):
            zo = ora.snr_at(j, o, g["t"].astype(np.int64))
            assert np.max(np.abs(np.sqrt(g["snr2"]) - np.abs(zo)) / np.abs(zo)) < EPS[rfd.PREC_FP16X3]
            checked += len(g)
    assert checked > 0
    assert compare_triggers(trig, sets, TOL_TC, sample, cfg.window) <= amb_cap(n_oracle(sets, sample))


# --------------------------------------------------------------------------- bucketed K (C3 shape)
def test_bucketed_taps_and_uneven_k_tensor_core(ctx):
    """Spin-orbit bank over 1-20 Msun on a 32 s / 2048 Hz grid: K_j chosen from the buckets
    32..512 by the ratio's bandwidth must equal the oracle's choice; lags and sigma_eff follow;
    the mixed-K bank filters in one tensor-core launch and matches the oracle's triggers."""
    from oracle import ratio
    cfg = workload.small_config(3, n=65536, n_tmpl=48, n_ref=4, threshold=9.0)
    bank, data = workload.make_workload(cfg)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    buckets = list(cfg.k_buckets)
    J = bank.n_tmpl
    taps = torch.zeros((J, 512), dtype=torch.complex64, device="cuda")
    lag = torch.zeros(J, dtype=torch.int32, device="cuda")
    sig = torch.zeros(J, dtype=torch.float64, device="cuda")
    kout = torch.zeros(J, dtype=torch.int32, device="cuda")
    rfd.make_taps(ctx, gpu.grid, gpu.psd, bank.ref_params(), bank.params(), bank.ref_of_tmpl, None, 512,
                  cfg.tukey_alpha, taps, lag, sig, buckets=buckets, energy_frac=0.999, k_out=kout)
    torch.cuda.synchronize()
    K = kout.cpu().numpy()
    lag_h, sig_h = lag.cpu().numpy(), sig.cpu().numpy()
    sets = {}
    for j in range(J):
        r = int(bank.ref_of_tmpl[j])
        G = ratio.ratio_spectrum(cfg.fs, cfg.n, cfg.f_low, bank.params()[j],
                                 bank.ref_params()[r], cfg.pn_flags)
        k_ora = ratio.k_bucket(ratio.impulse_response(G), buckets, 0.999)
        assert K[j] == k_ora, (j, K[j], k_ora)
        o = ora.design(j, int(K[j]), with_match=False)
        assert lag_h[j] == o["lag"], (j, lag_h[j], o["lag"])
        assert abs(sig_h[j] / o["sigma_eff"] - 1) < 1e-9
        sets[j] = ora.triggers(ora.snr(j, o), EPS[rfd.PREC_FP16X3])
    assert len(set(K.tolist())) >= 2                     # the bank really is uneven
    t = {"taps": taps, "lag": lag, "sigma": sig, "K": K.astype(np.int32), "k_stride": 512, "idx": np.arange(J)}
    q, e, _ = gpu.filter_reference(511, rfd.PREC_FP16X3)
    trig, ncand = gpu.ratio_filter(t, q, e, rfd.PREC_FP16X3, 511, cand_cap=1 << 22)
    n_or = n_oracle(sets, range(J))
    assert n_or > 50
    assert compare_triggers(trig, sets, TOL_TC, range(J), cfg.window) <= amb_cap(n_or)
    assert snr_errors(trig, sets, range(J)) < EPS[rfd.PREC_FP16X3]


# --------------------------------------------------------------------------- a very loud signal
@pytest.mark.parametrize("kernel,opts", TC_KERNELS)
def test_very_loud_injection_does_not_overflow_the_split(ctx, kernel, opts):
    """A 1024 s segment (n = 2^20 at 1024 Hz) with an injection at SNR 10^5 (standing for a
    very loud glitch or signal): its real part peaks 355 times above the rms of q_ref, past
    the FP16 range of a series scaled to an rms of 2^8 (65504 / 256 = 256 rms).  The split's
    scale is capped by the largest sample, so every trigger stays finite and matches the
    oracle (the many windows the loud chirp lights up included).  Rounding in FP32 (the
    reference's FFT, the accumulators) is relative to the largest values in flight, so here the
    error at each trigger is bounded by EPS times the template's peak |z|, and by the 1e-3
    target relative to the trigger's own |z|."""
    cfg = workload.small_config(1, n=1 << 20, inj_snr=(1e5, 1e5))
    bank, data = workload.make_workload(cfg)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP16X3)
    qo = ora.q_ref(0)
    rms = np.sqrt(np.mean(np.abs(qo) ** 2))
    assert max(np.max(np.abs(qo.real)), np.max(np.abs(qo.imag))) > 300 * rms
    assert int(e.item()) < 8 - int(np.log2(rms))           # the cap lowered the exponent
    trig, _ = gpu.ratio_filter(t, q, e, rfd.PREC_FP16X3, halo, cand_cap=1 << 22, options=opts)
    assert np.all(np.isfinite(trig["snr2"])) and np.all(np.isfinite(trig["zr"])) and np.all(np.isfinite(trig["zi"]))
    js = [0, 1, 2, 3, 17, 40]
    sets = {j: ora.triggers(ora.snr(j, ora.design(j, cfg.k, with_match=False)), EPS[rfd.PREC_FP16X3]) for j in js}
    n_or = n_oracle(sets, js)
    assert n_or > 20
    assert compare_triggers(trig, sets, TOL_TC, js, cfg.window) <= amb_cap(n_or)
    assert snr_errors(trig, sets, js) < TOL_TC
    for j in js:
        ot = {x["t"]: x["z"] for x in sets[j][0]}
        peak = max(abs(v) for v in ot.values())
        for r in trig[trig["j"] == j]:
            if int(r["t"]) in ot:
                zg = complex(float(r["zr"]), float(r["zi"]))
                assert abs(zg - ot[int(r["t"])]) <= EPS[rfd.PREC_FP16X3] * peak, (j, int(r["t"]))


# --------------------------------------------------------------------------- bounded waits
@pytest.mark.parametrize("kernel,opts", [("templates_on_m", {"long_k": 0}), ("time_on_m", {"long_k": 512})])
def test_bounded_wait_gives_up_and_the_context_stays_usable(c1, kernel, opts):
    """RFD_DEBUG_STALL_TAPS makes the tensor-core kernel never copy its taps, so the MMA
    thread's wait for them runs out (a short limit): the call reports RFD_ERR_TIMEOUT, every
    copy the producer did issue has landed before the CTAs end, and a normal call on the same
    context then succeeds and matches the oracle."""
    from paper_2601_18835_gb300 import _native
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP16X3)
    for _ in range(2):
        with pytest.raises(rfd.RfdError) as ei:
            gpu.ratio_filter(t, q, e, rfd.PREC_FP16X3, halo, options=dict(opts, debug_flags=_native.DEBUG_STALL_TAPS))
        assert ei.value.status == _native.RFD_ERR_TIMEOUT
    torch.cuda.synchronize()
    trig, _ = gpu.ratio_filter(t, q, e, rfd.PREC_FP16X3, halo, options=opts)
    sets = {j: ora.triggers(ora.snr(j, ora.design(j, cfg.k, with_match=False)), EPS[rfd.PREC_FP16X3])
            for j in range(bank.n_tmpl)}
    assert n_oracle(sets, range(bank.n_tmpl)) > 0
    assert compare_triggers(trig, sets, TOL_TC, range(bank.n_tmpl), cfg.window) <= amb_cap(
        n_oracle(sets, range(bank.n_tmpl)))
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[rfd.PREC_FP16X3]


# --------------------------------------------------------------------------- full series (Eq. 3)
# every kernel family in every precision: the FP32 CUDA-core FIR and the block-FFT kernel on an
# FP32 plan, and the three split-precision kernels (time on M, templates on M, block FFT)
SERIES_CASES = ([("fp32_direct", rfd.PREC_FP32, {}), ("fp32_block_fft", rfd.PREC_FP32, {"fft_k": 0})]
                + [("%s_%s" % (k, n), p, o) for (k, o) in TC_KERNELS for (n, p) in TC_PRECISIONS])


def series_error(ora, gpu, t, K, prec, opts, halo):
    """The GPU's whole SNR series (window 1, threshold 0: every sample is emitted) against the
    oracle's Eq. 3 series, template by template.  Returns the largest
    max_t |z_gpu[t] - z_oracle[t]| / rms_t |z_oracle|."""
    q, e, _ = gpu.filter_reference(halo, prec)
    zg, count = gpu.series(t, q, e, prec, halo, options=opts)
    worst, n_valid = 0.0, 0
    for j in range(len(K)):
        o = ora.design(j, int(K[j]), with_match=False)
        if o["sigma_eff"] == 0:
            assert not np.any(zg[j]), j          # all-zero taps (a 2-tap Tukey window): no output
            continue
        n_valid += 1
        zo = ora.snr(j, o)
        rms = np.sqrt(np.mean(np.abs(zo) ** 2))
        worst = max(worst, float(np.max(np.abs(zg[j] - zo)) / rms))
    assert count == n_valid * gpu.n              # every sample of every template, once
    return worst


@pytest.mark.parametrize("label,prec,opts", SERIES_CASES)
def test_full_series_c1(c1, label, prec, opts):
    """C1 (64 templates, K = 64): the whole series of every template."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    worst = series_error(ora, gpu, t, t["K"], prec, opts, cfg.k - 1)
    print("full series C1 %s: max |dz| / rms |z| = %.3g" % (label, worst))
    assert worst <= (TOL_FP32 if prec == rfd.PREC_FP32 else TOL_TC)
    assert worst <= EPS_SERIES[prec]


@pytest.mark.parametrize("label,prec,opts", SERIES_CASES)
def test_full_series_ragged(ctx, label, prec, opts):
    """37 templates (a ragged last tile), K from 2 to 96 (tiles padded to 16-tap steps; K = 2
    has all-zero Tukey taps): the whole series of every template."""
    cfg = workload.small_config(1, n_tmpl=37, window=37, threshold=6.0)
    bank, data = workload.make_workload(cfg)
    rng = np.random.default_rng(7)
    K = (2 * rng.integers(1, 49, size=bank.n_tmpl)).astype(np.int32)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=128, match=False)
    halo = int(((K.max() + 15) // 16) * 16) - 1
    worst = series_error(ora, gpu, t, K, prec, opts, halo)
    print("full series ragged %s: max |dz| / rms |z| = %.3g" % (label, worst))
    assert worst <= (TOL_FP32 if prec == rfd.PREC_FP32 else TOL_TC)
    assert worst <= EPS_SERIES[prec]


@pytest.mark.parametrize("name,prec", TC_PRECISIONS)
def test_full_series_tile_transitions_long_kernel(ctx, name, prec):
    """Templates-on-M kernel with tiles of one and two 64-tap chunks (taps resident for the
    tile) and of three and five chunks (streamed through the stages), interleaved along every
    CTA's range: 4 references x 4 K classes (no K mixing inside a tile), 16 tiles of 256 items.
    Five CTAs make each range cross resident -> resident, resident -> streamed, streamed ->
    streamed and streamed -> resident tile changes; one CTA crosses all of them in turn.  An
    item's arithmetic does not depend on which CTA runs it, so the whole series must be
    bit-identical across the partitions; against the oracle, every sample lies within the
    path's bound of the series' peak (the bank carries loud injections, so the rms is far
    below the peak) and within the method's 1e-3 of its rms."""
    cfg = workload.small_config(3, n=65536, n_tmpl=32, n_ref=4)
    bank, data = workload.make_workload(cfg)
    classes = np.array([48, 128, 192, 320], dtype=np.int32)
    K = np.zeros(bank.n_tmpl, dtype=np.int32)
    for r in range(bank.n_ref):                          # the K classes in turn within each reference
        members = np.flatnonzero(bank.ref_of_tmpl == r)
        K[members] = classes[np.arange(len(members)) % 4]
    for r in range(bank.n_ref):                          # every reference holds every K class
        assert set(K[bank.ref_of_tmpl == r].tolist()) == {48, 128, 192, 320}
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=320, match=False)
    opts = {"long_k": 0, "mix_k": 0, "grid_ctas": 5}
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, K, prec, cfg.window, cfg.threshold, 319,
                    options=opts)
    kinds = plan.template_kernels()
    plan.close()
    assert np.all(kinds == 2)                            # every template on the templates-on-M kernel
    q, e, _ = gpu.filter_reference(319, prec)
    z5, count = gpu.series(t, q, e, prec, 319, options=opts)
    assert count == bank.n_tmpl * gpu.n                  # every sample of every template, once
    z1, _ = gpu.series(t, q, e, prec, 319, options=dict(opts, grid_ctas=1))
    zd, _ = gpu.series(t, q, e, prec, 319, options={"long_k": 0, "mix_k": 0})
    assert np.array_equal(z5, z1) and np.array_equal(z5, zd)
    worst_rms = worst_peak = 0.0
    for j in range(bank.n_tmpl):
        zo = ora.snr(j, ora.design(j, int(K[j]), with_match=False))
        d = float(np.max(np.abs(z5[j] - zo)))
        worst_rms = max(worst_rms, d / float(np.sqrt(np.mean(np.abs(zo) ** 2))))
        worst_peak = max(worst_peak, d / float(np.max(np.abs(zo))))
    print("full series tile transitions %s: max |dz| / rms |z| = %.3g, / peak |z| = %.3g" % (name, worst_rms,
                                                                                             worst_peak))
    assert worst_rms <= TOL_TC
    assert worst_peak <= EPS[prec]


# --------------------------------------------------------------------------- graph and autotuner
@pytest.mark.parametrize("opts", [None, {"fft_k": 32}])
def test_search_graph_matches_separate_calls(c1, opts):
    """The whole segment as one CUDA graph (rfd_search_*) equals the three separate calls, on two
    segments in a row (the second written into the bound spectrum buffer); also with the
    block-FFT kernel in the plan."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    href = gpu.templates(bank.ref_params())
    ld = rfd.qref_ld(cfg.n, halo)
    q = torch.zeros(bank.n_ref * ld * 8, dtype=torch.uint8, device="cuda")
    e = torch.zeros(bank.n_ref, dtype=torch.int32, device="cuda")
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], rfd.PREC_FP16X3, cfg.window,
                    cfg.threshold, halo, options=opts)
    plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
    cap, tcap = 1 << 18, 1 << 16
    cand = torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    trig = torch.zeros(tcap * 20, dtype=torch.uint8, device="cuda")
    d = gpu.d.clone()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        search = rfd.Search(plan, d, gpu.psd, href, q, e, cand, cnt, trig, stream)
    assert search.kernels_per_run >= 8
    rng = np.random.default_rng(3)
    for seg in range(2):
        if seg:
            noise = (rng.standard_normal(d.numel()) + 1j * rng.standard_normal(d.numel())).astype(np.complex64)
            d.copy_(torch.from_numpy(noise * np.abs(data.dtilde.astype(np.complex64))))
        torch.cuda.synchronize()
        nt_graph = search.run()
        got = rfd.triggers_to_numpy(trig, nt_graph).copy()
        # the same segment through the separate calls
        rfd.filter_reference(gpu.ctx, gpu.grid, d, gpu.psd, href, halo, rfd.PREC_FP16X3, q, e)
        plan.ratio_filter_batch(q, e, cand, cnt)
        trig2 = torch.zeros_like(trig)
        nt2 = rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, trig2)
        assert nt_graph == nt2
        assert np.array_equal(got.view(np.uint8), rfd.triggers_to_numpy(trig2, nt2).view(np.uint8))
    search.close()
    plan.close()


def test_search_survives_scratch_growth(c1):
    """A call that needs larger context scratch buffers after the graph was captured (here a
    filter_reference over four times as many references) leaves the graph's buffers valid:
    the next replay gives the same triggers as before."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    href = gpu.templates(bank.ref_params())
    ld = rfd.qref_ld(cfg.n, halo)
    q = torch.zeros(bank.n_ref * ld * 8, dtype=torch.uint8, device="cuda")
    e = torch.zeros(bank.n_ref, dtype=torch.int32, device="cuda")
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], rfd.PREC_FP16X3, cfg.window,
                    cfg.threshold, halo)
    plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
    cand = torch.zeros((1 << 18) * 24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    trig = torch.zeros((1 << 16) * 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        search = rfd.Search(plan, gpu.d, gpu.psd, href, q, e, cand, cnt, trig, stream)
    n0 = search.run()
    before = rfd.triggers_to_numpy(trig, n0).view(np.uint8).copy()
    R4 = 4 * bank.n_ref + 3
    href4 = href.repeat(R4, 1)[:R4].contiguous()
    q4 = torch.zeros(R4 * ld * 8, dtype=torch.uint8, device="cuda")
    e4 = torch.zeros(R4, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        rfd.filter_reference(gpu.ctx, gpu.grid, gpu.d, gpu.psd, href4, halo, rfd.PREC_FP16X3, q4, e4, stream=stream)
    stream.synchronize()
    n1 = search.run()
    assert n1 == n0
    assert np.array_equal(rfd.triggers_to_numpy(trig, n1).view(np.uint8), before)
    search.close()
    plan.close()


WINDOW_KERNELS = [("fp32", 0, {}), ("time_on_m", 1, {"long_k": 512}), ("templates_on_m", 1, {"long_k": 0}),
                  ("block_fft", 1, {"fft_k": 0})]


def _merge_windows(trig_list, window):
    """Per (j, t // window) the trigger with the largest |z|^2 (ties: smallest t) over the
    windows' trigger lists, as find_triggers merges candidates."""
    best = {}
    for tr in trig_list:
        for x in tr:
            key = (int(x["j"]), int(x["t"]) // window)
            cur = best.get(key)
            if cur is None or (x["snr2"], -int(x["t"])) > (cur["snr2"], -int(cur["t"])):
                best[key] = x
    return best


@pytest.mark.parametrize("kernel,prec,opts", WINDOW_KERNELS)
def test_windows_tile_the_segment(c1, kernel, prec, opts):
    """Streaming (out_len = 2048 of n = 16384): the eight windows' candidates, merged by
    find_triggers, give the full-segment triggers (bit for bit on the direct kernels; the
    block-FFT kernel cuts its blocks at each window start, so there SNRs agree to 1e-5)."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, prec)
    full, _ = gpu.ratio_filter(t, q, e, prec, halo, options=opts)
    B = 2048
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], prec, cfg.window, cfg.threshold, halo,
                    options=dict(opts, out_len=B))
    plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
    cap = 1 << 16
    parts, total = [], 0
    u = torch.zeros(1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for w0 in range(0, cfg.n, B):
        cand = torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
        u.fill_(w0)
        plan.ratio_filter_window(q, e, u, cand, cnt)
        nc = int(cnt.item())
        assert nc < cap
        parts.append(cand[: nc * 24].clone())
        total += nc
    plan.close()
    allc = torch.cat(parts) if total else torch.zeros(24, dtype=torch.uint8, device="cuda")
    cnt.fill_(total)
    tb = torch.zeros((1 << 16) * 20, dtype=torch.uint8, device="cuda")
    nt = rfd.find_triggers(gpu.ctx, bank.n_tmpl, allc, cnt, tb)
    got = rfd.triggers_to_numpy(tb, nt)
    assert len(full) > 0
    if kernel != "block_fft":
        assert np.array_equal(got.view(np.uint8), full.view(np.uint8))
    else:
        a = {(int(x["j"]), int(x["t"]) // cfg.window): x for x in full}
        b = {(int(x["j"]), int(x["t"]) // cfg.window): x for x in got}
        assert len(set(a) ^ set(b)) <= 2
        for key in set(a) & set(b):
            assert abs(math.sqrt(float(a[key]["snr2"])) / math.sqrt(float(b[key]["snr2"])) - 1) < 1e-5


def test_streaming_search_graph(c1):
    """A captured search on a window plan, replayed at each window start (rfd_search_run_at):
    the windows' triggers merged per (template, window) equal the full-segment search's."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    href = gpu.templates(bank.ref_params())
    ld = rfd.qref_ld(cfg.n, halo)
    stream = torch.cuda.Stream()
    out = []
    for out_len in (0, 2048):
        q = torch.zeros(bank.n_ref * ld * 8, dtype=torch.uint8, device="cuda")
        e = torch.zeros(bank.n_ref, dtype=torch.int32, device="cuda")
        plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], rfd.PREC_FP16X3, cfg.window,
                        cfg.threshold, halo, options={"out_len": out_len})
        plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
        cand = torch.zeros((1 << 18) * 24, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        trig = torch.zeros((1 << 16) * 20, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(stream):
            search = rfd.Search(plan, gpu.d, gpu.psd, href, q, e, cand, cnt, trig, stream)
        lists = []
        for w0 in (range(0, cfg.n, out_len) if out_len else [0]):
            nt = search.run(u_begin=w0)
            lists.append(rfd.triggers_to_numpy(trig, nt).copy())
        out.append(_merge_windows(lists, cfg.window))
        search.close()
        plan.close()
    full, win = out
    assert len(full) > 0 and set(full) == set(win)
    for key in full:
        assert full[key].tobytes() == win[key].tobytes()


def test_autotuner_choices_give_identical_triggers(ctx, tmp_path):
    """Every tile choice the autotuner tries gives bit-identical triggers (tiles only change
    which templates share an MMA and how many zero taps pad them); the tuner caches its pick."""
    from paper_2601_18835_gb300 import autotune
    cfg = workload.small_config(3, n=65536, n_tmpl=96, n_ref=3, threshold=9.0)
    bank, data = workload.make_workload(cfg)
    gpu = GpuRun(cfg, bank, data, ctx=ctx)
    J = bank.n_tmpl
    taps = torch.zeros((J, 512), dtype=torch.complex64, device="cuda")
    lag = torch.zeros(J, dtype=torch.int32, device="cuda")
    sig = torch.zeros(J, dtype=torch.float64, device="cuda")
    kout = torch.zeros(J, dtype=torch.int32, device="cuda")
    rfd.make_taps(ctx, gpu.grid, gpu.psd, bank.ref_params(), bank.params(), bank.ref_of_tmpl, None, 512,
                  cfg.tukey_alpha, taps, lag, sig, buckets=list(cfg.k_buckets), k_out=kout)
    K = kout.cpu().numpy().astype(np.int32)
    q, e, _ = gpu.filter_reference(511, rfd.PREC_FP16X3)
    cache = str(tmp_path / "tune.json")
    opts, rep = autotune.autotune(ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, K, rfd.PREC_FP16X3, cfg.window,
                                  cfg.threshold, 511, taps, 512, lag, sig, q, e, cache_path=cache)
    assert opts in [c["options"] for c in rep["candidates"]]
    opts2, rep2 = autotune.autotune(ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, K, rfd.PREC_FP16X3, cfg.window,
                                    cfg.threshold, 511, taps, 512, lag, sig, q, e, cache_path=cache)
    assert opts2 == opts
    results = []
    for c in rep["candidates"]:
        plan = rfd.Plan(ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, K, rfd.PREC_FP16X3, cfg.window, cfg.threshold,
                        511, options=c["options"])
        plan.set_taps(taps, 512, lag, sig)
        cand = torch.zeros((1 << 22) * 24, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        plan.ratio_filter_batch(q, e, cand, cnt)
        tb = torch.zeros((1 << 18) * 20, dtype=torch.uint8, device="cuda")
        nt = rfd.find_triggers(ctx, J, cand, cnt, tb)
        results.append(rfd.triggers_to_numpy(tb, nt).view(np.uint8).copy())
        plan.close()
    assert len(results[0]) > 0
    # tensor-core choices: bit-identical; block-FFT choices (other arithmetic): the same windows
    # and samples, |z| within the tensor-core tolerance
    base = results[0].view(rfd.TRIGGER_DTYPE)
    for c, r in zip(rep["candidates"][1:], results[1:]):
        if "fft_k" not in c["options"] and "fft_rem" not in c["options"]:
            assert np.array_equal(r, results[0])
            continue
        got = r.view(rfd.TRIGGER_DTYPE)
        a = {(int(x["j"]), int(x["t"]) // cfg.window): x for x in base}
        b = {(int(x["j"]), int(x["t"]) // cfg.window): x for x in got}
        diff = set(a) ^ set(b)
        assert len(diff) <= 0.01 * len(a), (c["options"], len(diff))
        for key in set(a) & set(b):
            za, zb = math.sqrt(float(a[key]["snr2"])), math.sqrt(float(b[key]["snr2"]))
            assert abs(za - zb) <= 2e-3 * za, (c["options"], key, za, zb)


def test_search_graph_times_each_run(c1):
    """The events inside the graph are re-recorded on every replay: after two runs, two
    different, positive step times, each longer than the ratio-filter kernel inside it."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    href = gpu.templates(bank.ref_params())
    ld = rfd.qref_ld(cfg.n, halo)
    q = torch.zeros(bank.n_ref * ld * 8, dtype=torch.uint8, device="cuda")
    e = torch.zeros(bank.n_ref, dtype=torch.int32, device="cuda")
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], rfd.PREC_FP16X3, cfg.window,
                    cfg.threshold, halo)
    plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
    cand = torch.zeros((1 << 16) * 24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    trig = torch.zeros((1 << 14) * 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        search = rfd.Search(plan, gpu.d, gpu.psd, href, q, e, cand, cnt, trig, stream)
    times = []
    for _ in range(3):
        search.run()
        step, kern = search.step_ms(), search.filter_ms()
        assert 0 < kern < step
        times.append(step)
    assert len(set(times)) > 1
    # nothing left behind for the next call's error check
    rfd.filter_reference(gpu.ctx, gpu.grid, gpu.d, gpu.psd, href, halo, rfd.PREC_FP16X3, q, e)
    search.close()
    plan.close()

"""Edge cases of the ratio-filter path (Eq. 3 and the trigger reduction) on the GPU, each against
the FP64 oracle or an exact count:

* nothing over the threshold, with zero-capacity candidate and trigger lists;
* single-tap templates (K = 1) next to K = 16, 17 and 64, with a reference that holds no
  template, for every kernel family in every precision (the whole series);
* a trigger window longer than the segment (one trigger per template: its whole-series maximum);
* the largest grid the library accepts, n = 2^22, end to end with the oracle on a sample.
"""
import dataclasses

import numpy as np
import pytest

import workload
from oracle import triggers as otrig
from tests.oracle_pipeline import OracleRun

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402
from tests.gpu_pipeline import GpuRun  # noqa: E402
from tests.test_gpu_parity import (EPS, EPS_SERIES, SERIES_CASES, TOL_FP32, TOL_TC, amb_cap,  # noqa: E402
                                   compare_triggers, n_oracle, series_error)

# (name, precision, plan options, the kernel every template must land on: 0 FP32 direct FIR,
# 1 tensor cores with time on M, 2 tensor cores with templates on M, 3 block FFT)
FAMILIES = [("fp32_fir", rfd.PREC_FP32, {}, 0),
            ("tc_time_on_m", rfd.PREC_FP16X3, {"long_k": 512}, 1),
            ("tc_templates_on_m", rfd.PREC_FP16X3, {"long_k": 0, "fft_rem": 0}, 2),
            ("block_fft", rfd.PREC_FP16X3, {"fft_k": 0}, 3)]


@pytest.fixture(scope="module")
def ctx():
    c = rfd.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def c1(ctx):
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg)
    return cfg, bank, data, OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)


def tol_of(prec):
    return TOL_FP32 if prec == rfd.PREC_FP32 else TOL_TC


@pytest.mark.parametrize("name,prec,opts,kernel", FAMILIES)
def test_nothing_over_the_threshold(c1, name, prec, opts, kernel):
    """A threshold no sample reaches: no candidate, no trigger, no overflow, even with lists of
    capacity zero."""
    cfg, bank, data, ora, gpu = c1
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, prec)
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], prec, cfg.window, 1e30, halo,
                    options=opts)
    try:
        assert set(plan.template_kernels().tolist()) == {kernel}
        plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
        empty = torch.zeros(0, dtype=torch.uint8, device="cuda")
        cnt = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
        plan.ratio_filter_batch(q, e, empty, cnt)
        assert int(cnt.item()) == 0
        assert rfd.find_triggers(gpu.ctx, bank.n_tmpl, empty, cnt, empty) == 0
    finally:
        plan.close()


@pytest.fixture(scope="module")
def single_tap_bank():
    """24 templates over 3 references, reference 1's templates moved to the nearest other
    reference (so that reference holds none); K cycles through 1, 16, 17, 64."""
    cfg = workload.small_config(1, n_tmpl=24, n_ref=3, c1_slots=False, window=64, threshold=6.0)
    bank, data = workload.make_workload(cfg)
    mc = workload.chirp_mass(bank.m1, bank.m2)
    ref_mc = workload.chirp_mass(bank.ref_m1, bank.ref_m2)
    ref_of = bank.ref_of_tmpl.copy()
    moved = ref_of == 1
    assert moved.any()
    ref_of[moved] = np.where(np.abs(mc[moved] - ref_mc[0]) <= np.abs(mc[moved] - ref_mc[2]), 0, 2)
    bank = dataclasses.replace(bank, ref_of_tmpl=ref_of.astype(np.int32))
    assert set(bank.ref_of_tmpl.tolist()) == {0, 2}
    K = np.array([1, 16, 17, 64], dtype=np.int32)[np.arange(bank.n_tmpl) % 4]
    return cfg, bank, data, K


@pytest.mark.parametrize("label,prec,opts", SERIES_CASES)
def test_single_taps_and_an_unused_reference(ctx, single_tap_bank, label, prec, opts):
    cfg, bank, data, K = single_tap_bank
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(K, k_stride=64, match=False)
    worst = series_error(ora, gpu, t, K, prec, opts, 63)
    print("full series single taps %s: max |dz| / rms |z| = %.3g" % (label, worst))
    assert worst <= tol_of(prec)
    assert worst <= EPS_SERIES[prec]


@pytest.mark.parametrize("name,prec,opts,kernel", FAMILIES)
def test_window_longer_than_the_segment(c1, name, prec, opts, kernel):
    """W = n + 123: every template's one window covers the whole segment, so its trigger is the
    maximum of its whole series (when that clears the threshold)."""
    cfg, bank, data, ora, gpu = c1
    W = gpu.n + 123
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, prec)
    trig, _ = gpu.ratio_filter(t, q, e, prec, halo, options=opts, window=W)
    sets = {}
    for j in range(bank.n_tmpl):
        z = ora.snr(j, ora.design(j, cfg.k, with_match=False))
        sets[j] = otrig.window_triggers(z, W, cfg.threshold, tol=EPS[prec])
        assert len(sets[j][0]) <= 1
    assert len(trig) == n_oracle(sets, range(bank.n_tmpl)) and np.all(np.diff(trig["j"]) > 0)
    assert compare_triggers(trig, sets, tol_of(prec), range(bank.n_tmpl), W) <= amb_cap(
        n_oracle(sets, range(bank.n_tmpl)))


@pytest.mark.slow
def test_largest_grid(ctx):
    """n = 2^22 (4096 s at 1024 Hz), the largest grid the library accepts: 8 templates over 2
    references, K = 32, every kernel family; the oracle's whole series for the injected template
    and one template per reference, and every GPU trigger of those re-evaluated at its sample."""
    cfg = workload.small_config(1, n=1 << 22, n_tmpl=8, n_ref=2, c1_slots=False, k=32)
    bank, data = workload.make_workload(cfg)
    ora, gpu = OracleRun(cfg, bank, data), GpuRun(cfg, bank, data, ctx=ctx)
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    sample = sorted({s for (_, _, _, s) in data.injections}
                    | {int(np.nonzero(bank.ref_of_tmpl == r)[0][0]) for r in range(bank.n_ref)})
    designs = {j: ora.design(j, cfg.k, with_match=False) for j in sample}
    series = {j: ora.snr(j, designs[j]) for j in sample}
    for name, prec, opts, kernel in FAMILIES:
        q, e, _ = gpu.filter_reference(halo, prec)
        trig, _ = gpu.ratio_filter(t, q, e, prec, halo, cand_cap=1 << 22, options=opts)
        sets, checked = {}, 0
        for j in sample:
            sets[j] = ora.triggers(series[j], EPS[prec])
            g = trig[trig["j"] == j]
            if len(g):
                zo = ora.snr_at(j, designs[j], g["t"].astype(np.int64))
                assert np.max(np.abs(np.sqrt(g["snr2"]) - np.abs(zo)) / np.abs(zo)) < EPS[prec], name
                checked += len(g)
        assert checked > 0, name
        assert compare_triggers(trig, sets, tol_of(prec), sample, cfg.window) <= amb_cap(
            n_oracle(sets, sample)), name

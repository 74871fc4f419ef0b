"""Determinism and guard canaries: the repository's substitute for a race detector, which this
pool does not offer.

* Ten runs of the same plan on the same inputs give byte-identical candidate counts and
  trigger lists, for every kernel family (the trigger merge uses integer keys only, so any
  nondeterminism in a kernel would show up here).
* No call writes past the capacity it was given: the candidate list, the trigger list and the
  reference series are each passed as a view of a larger allocation whose tail holds a byte
  pattern, and the tail is unchanged afterwards; also when the candidate list overflows.
"""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402
import workload  # noqa: E402
from tests.gpu_pipeline import GpuRun  # noqa: E402

CANARY = 0xA5
RFD_ERR_OVERFLOW = -7
# (name, precision, plan options, the kernel every template must land on: 0 FP32 direct FIR,
# 1 tensor cores with time on M, 2 tensor cores with templates on M, 3 block FFT)
FAMILIES = [("fp32_fir", rfd.PREC_FP32, {}, 0),
            ("tc_time_on_m", rfd.PREC_FP16X3, {"long_k": 512}, 1),
            ("tc_templates_on_m", rfd.PREC_FP16X3, {"long_k": 0, "fft_rem": 0}, 2),
            ("block_fft", rfd.PREC_FP16X3, {"fft_k": 0}, 3)]


@pytest.fixture(scope="module")
def case():
    cfg = workload.small_config(1, n_tmpl=48, threshold=9.0)
    bank, data = workload.make_workload(cfg)
    gpu = GpuRun(cfg, bank, data)
    t = gpu.make_taps(cfg.k, match=False)
    return cfg, bank, gpu, t


def guarded(nbytes, tail=4096):
    """A uint8 tensor of nbytes whose storage continues for `tail` canary bytes."""
    buf = torch.full((nbytes + tail,), CANARY, dtype=torch.uint8, device="cuda")
    return buf, buf[:nbytes]


def tail_intact(buf, nbytes):
    return bool(torch.all(buf[nbytes:] == CANARY).item())


def make_plan(cfg, bank, gpu, t, prec, opts, kernel):
    plan = rfd.Plan(gpu.ctx, gpu.grid, bank.n_ref, bank.ref_of_tmpl, t["K"], prec, cfg.window, cfg.threshold,
                    cfg.k - 1, options=opts)
    assert set(plan.template_kernels().tolist()) == {kernel}
    plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
    return plan


@pytest.mark.parametrize("name,prec,opts,kernel", FAMILIES)
def test_ten_runs_identical(case, name, prec, opts, kernel):
    cfg, bank, gpu, t = case
    q, e, _ = gpu.filter_reference(cfg.k - 1, prec)
    plan = make_plan(cfg, bank, gpu, t, prec, opts, kernel)
    try:
        cand = torch.zeros((1 << 16) * 24, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        trig = torch.zeros((1 << 14) * 20, dtype=torch.uint8, device="cuda")
        ref = None
        for run in range(10):
            plan.ratio_filter_batch(q, e, cand, cnt)
            nt = rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, trig)
            got = (int(cnt.item()), rfd.triggers_to_numpy(trig, nt).tobytes())
            assert got[0] > 0 and nt > 0
            if ref is None:
                ref = got
            assert got == ref, (name, run)
    finally:
        plan.close()


@pytest.mark.parametrize("name,prec,opts,kernel", FAMILIES)
def test_no_write_past_capacity(case, name, prec, opts, kernel):
    cfg, bank, gpu, t = case
    halo = cfg.k - 1
    # the reference series: exactly the documented size (8 bytes a sample in every precision:
    # complex64, or four 16-bit planes), then the canary
    R, ld = bank.n_ref, rfd.qref_ld(gpu.n, halo)
    qbytes = R * ld * 8
    qbuf, q = guarded(qbytes)
    e = torch.zeros(R, dtype=torch.int32, device="cuda")
    href = gpu.templates(bank.ref_params())
    rfd.filter_reference(gpu.ctx, gpu.grid, gpu.d, gpu.psd, href, halo, prec, q, e)
    torch.cuda.synchronize()
    assert tail_intact(qbuf, qbytes)
    plan = make_plan(cfg, bank, gpu, t, prec, opts, kernel)
    try:
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        # enough room: every candidate fits, the tail stays untouched
        cbuf, cand = guarded((1 << 16) * 24)
        plan.ratio_filter_batch(q, e, cand, cnt)
        torch.cuda.synchronize()
        n_cand = int(cnt.item())
        assert 0 < n_cand < (1 << 16) and tail_intact(cbuf, (1 << 16) * 24)
        # the trigger list: exactly as many records as there are triggers, then the canary
        probe = torch.zeros((1 << 14) * 20, dtype=torch.uint8, device="cuda")
        n_trig = rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, probe)
        assert n_trig > 0
        tbuf, trig = guarded(n_trig * 20)
        assert rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, trig) == n_trig
        torch.cuda.synchronize()
        assert tail_intact(tbuf, n_trig * 20)
        if n_trig > 1:                                 # one record short: reported, nothing written past it
            tbuf, trig = guarded((n_trig - 1) * 20)
            with pytest.raises(rfd.RfdError) as err:
                rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, trig)
            torch.cuda.synchronize()
            assert err.value.status == RFD_ERR_OVERFLOW and err.value.needed == n_trig
            assert tail_intact(tbuf, (n_trig - 1) * 20)
        # too little room: the overflow is reported with the count, and nothing lands past it
        small = max(1, n_cand // 3)
        sbuf, scand = guarded(small * 24)
        plan.ratio_filter_batch(q, e, scand, cnt)
        torch.cuda.synchronize()
        assert int(cnt.item()) == n_cand and tail_intact(sbuf, small * 24)
        with pytest.raises(rfd.RfdError) as err:
            rfd.find_triggers(gpu.ctx, bank.n_tmpl, scand, cnt, probe)
        assert err.value.status == RFD_ERR_OVERFLOW and err.value.needed == n_cand
    finally:
        plan.close()

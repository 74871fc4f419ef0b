"""rfd_find_triggers_noalloc against rfd_find_triggers.

The no-allocation variant exists for callers that cannot allocate device memory once they
run (allocation can synchronise the whole device, or their memory belongs to another
allocator).  It keeps its scratch in a fixed static device array.  Here it is called through
the C ABI twice in a row, on two different candidate lists, and each result must equal what
the allocating entry point returns for the same candidates.  The merge is integer-only, so
the comparison is exact.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402
from tests.gpu_pipeline import GpuRun  # noqa: E402


def candidates(gpu, threshold, cap):
    """Run the FP32 ratio filter on the C1 workload with `threshold`; return (cand, count)."""
    cfg = gpu.cfg
    t = gpu.make_taps(cfg.k, match=False)
    halo = cfg.k - 1
    q, e, _ = gpu.filter_reference(halo, rfd.PREC_FP32)
    plan = rfd.Plan(gpu.ctx, gpu.grid, gpu.bank.n_ref, gpu.bank.ref_of_tmpl, t["K"], rfd.PREC_FP32, cfg.window,
                    threshold, halo)
    plan.set_taps(t["taps"], t["k_stride"], t["lag"], t["sigma"])
    cand = torch.zeros(cap * 24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    plan.ratio_filter_batch(q, e, cand, cnt)
    torch.cuda.synchronize()
    plan.close()
    return cand, cnt


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    from paper_2601_18835_gb300 import build
    build.build()
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg)
    gpu = GpuRun(cfg, bank, data)
    cap = 1 << 16
    results = []
    for thr in (25.0, 9.0):                      # two different candidate lists, one after the other
        cand, cnt = candidates(gpu, thr, cap)
        assert 0 < int(cnt.item()) <= cap
        ref_buf = torch.zeros((1 << 15) * 20, dtype=torch.uint8, device="cuda")
        n_ref = rfd.find_triggers(gpu.ctx, bank.n_tmpl, cand, cnt, ref_buf)
        na_buf = torch.full(((1 << 15) * 20,), 0xAB, dtype=torch.uint8, device="cuda")
        n_na = rfd.find_triggers_noalloc(bank.n_tmpl, cand, cnt, na_buf)
        assert n_na == n_ref
        a = ref_buf[: n_ref * 20].cpu().numpy()
        b = na_buf[: n_na * 20].cpu().numpy()
        assert np.array_equal(a, b)
        results.append(n_ref)
    assert results[1] > results[0]              # the lower threshold gives more triggers


def test_noalloc_rejects_sizes_beyond_its_maximum():
    from paper_2601_18835_gb300 import _native
    cand = torch.zeros(24, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    trig = torch.zeros(20, dtype=torch.uint8, device="cuda")
    with pytest.raises(rfd.RfdError) as ei:
        rfd.find_triggers_noalloc(_native.NOALLOC_MAX_TEMPLATES + 1, cand, cnt, trig)
    assert ei.value.status == _native.RFD_ERR_SHAPE
    big = torch.zeros((_native.NOALLOC_MAX_CANDIDATES + 1) * 24, dtype=torch.uint8, device="cuda")
    with pytest.raises(rfd.RfdError) as ei:
        rfd.find_triggers_noalloc(4, big, cnt, trig)
    assert ei.value.status == _native.RFD_ERR_SHAPE


def test_noalloc_allocates_nothing_and_leaves_no_stale_state():
    """After a first call has loaded the module (set-up), a further call changes the device's
    free memory by nothing; and a call with fewer templates and candidates than the call
    before it (so the static array still holds the larger call's words past its own) equals
    the allocating entry point on the same list."""
    from tests.test_gpu_triggers import synthetic_candidates
    ctx = rfd.Context(0)
    W = 37
    outs = []
    for seed, n_tmpl in ((5, 60), (6, 12)):
        rng = np.random.default_rng(seed)
        recs = synthetic_candidates(rng, n_tmpl, W)
        cand = np.zeros(len(recs), dtype=rfd.CANDIDATE_DTYPE)
        for i, (j, t, p) in enumerate(recs):
            cand[i]["key"] = (int(np.float32(p).view(np.uint32)) << 32) | (0xFFFFFFFF - t)
            cand[i]["j"], cand[i]["w"], cand[i]["zr"], cand[i]["zi"] = j, t // W, np.sqrt(p), t
        cd = torch.from_numpy(cand.view(np.uint8).copy()).cuda()
        cnt = torch.tensor([len(recs)], dtype=torch.int64, device="cuda")
        ref_buf = torch.zeros((1 << 16) * 20, dtype=torch.uint8, device="cuda")
        n_ref = rfd.find_triggers(ctx, n_tmpl, cd, cnt, ref_buf)
        na_buf = torch.full(((1 << 16) * 20,), 0xAB, dtype=torch.uint8, device="cuda")
        n_first = rfd.find_triggers_noalloc(n_tmpl, cd, cnt, na_buf)     # right after the other list
        assert n_first == n_ref
        assert np.array_equal(ref_buf[: n_ref * 20].cpu().numpy(), na_buf[: n_first * 20].cpu().numpy())
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        na_buf.fill_(0xAB)
        n_na = rfd.find_triggers_noalloc(n_tmpl, cd, cnt, na_buf)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert n_na == n_ref
        assert np.array_equal(ref_buf[: n_ref * 20].cpu().numpy(), na_buf[: n_na * 20].cpu().numpy())
        outs.append(n_ref)
    assert outs[1] < outs[0]
    ctx.close()

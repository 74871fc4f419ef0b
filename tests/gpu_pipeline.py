"""GPU side of the parity tests: the ratio-filter path through the librfd C ABI only."""
import numpy as np
import torch

import paper_2601_18835_gb300 as rfd


class GpuRun:
    def __init__(self, cfg, bank, data, n=None, ctx=None):
        self.cfg = cfg
        self.bank = bank
        self.n = cfg.n if n is None else n
        self.ctx = ctx or rfd.Context(0)
        self.grid = rfd.grid(cfg.fs, self.n, cfg.f_low, cfg.pn_flags)
        self.psd = torch.from_numpy(data.psd).cuda()
        self.d = torch.from_numpy(data.dtilde.astype(np.complex64)).cuda()

    def make_taps(self, K, k_stride=None, match=True, tmpl_idx=None):
        idx = np.arange(self.bank.n_tmpl) if tmpl_idx is None else np.asarray(tmpl_idx)
        K = np.broadcast_to(np.asarray(K, dtype=np.int32), idx.shape).copy()
        ks = int(k_stride or K.max())
        J = len(idx)
        taps = torch.zeros((J, ks), dtype=torch.complex64, device="cuda")
        lag = torch.zeros(J, dtype=torch.int32, device="cuda")
        sig = torch.zeros(J, dtype=torch.float64, device="cuda")
        mat = torch.zeros(J, dtype=torch.float64, device="cuda") if match else None
        rfd.make_taps(self.ctx, self.grid, self.psd, self.bank.ref_params(), self.bank.params()[idx],
                      self.bank.ref_of_tmpl[idx], K, ks, self.cfg.tukey_alpha, taps, lag, sig, mat)
        torch.cuda.synchronize()
        return {"taps": taps, "lag": lag, "sigma": sig, "match": mat, "K": K, "k_stride": ks, "idx": idx}

    def templates(self, params):
        h = torch.zeros((len(params), self.n // 2 + 1), dtype=torch.complex64, device="cuda")
        rfd.gen_templates(self.ctx, self.grid, params, h)
        return h

    def filter_reference(self, halo, precision):
        R = self.bank.n_ref
        ld = rfd.qref_ld(self.n, halo)
        q = torch.zeros(R * ld * 8, dtype=torch.uint8, device="cuda")
        e = torch.zeros(R, dtype=torch.int32, device="cuda")
        href = self.templates(self.bank.ref_params())
        rfd.filter_reference(self.ctx, self.grid, self.d, self.psd, href, halo, precision, q, e)
        torch.cuda.synchronize()
        return q, e, ld

    def ratio_filter(self, taps, q, e, precision, halo, cand_cap=1 << 20, trig_cap=1 << 18, options=None,
                     window=None, threshold=None):
        idx = taps["idx"]
        W = self.cfg.window if window is None else window
        thr = self.cfg.threshold if threshold is None else threshold
        plan = rfd.Plan(self.ctx, self.grid, self.bank.n_ref, self.bank.ref_of_tmpl[idx], taps["K"], precision,
                        W, thr, halo, options=options)
        try:
            plan.set_taps(taps["taps"], taps["k_stride"], taps["lag"], taps["sigma"])
            cand = torch.zeros(cand_cap * 24, dtype=torch.uint8, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            plan.ratio_filter_batch(q, e, cand, cnt)
            trig = torch.zeros(trig_cap * 20, dtype=torch.uint8, device="cuda")
            nt = rfd.find_triggers(self.ctx, len(idx), cand, cnt, trig)
            out = rfd.triggers_to_numpy(trig, nt).copy()
            ncand = int(cnt.item())
        finally:
            plan.close()
        return out, ncand

    def series(self, taps, q, e, precision, halo, options=None):
        """The whole SNR series of every template through the production kernels: window 1 and
        threshold 0 make every sample with |z|^2 > 0 its own trigger.  Returns complex z[J, n]
        (zero where nothing was emitted) and the number of (j, t) emitted."""
        J = len(taps["idx"])
        cap = J * self.n + 1024
        trig, ncand = self.ratio_filter(taps, q, e, precision, halo, cand_cap=cap, trig_cap=cap, options=options,
                                        window=1, threshold=0.0)
        z = np.zeros((J, self.n), dtype=np.complex128)
        z[trig["j"].astype(np.int64), trig["t"].astype(np.int64)] = trig["zr"].astype(np.float64) + \
            1j * trig["zi"].astype(np.float64)
        return z, len(trig)

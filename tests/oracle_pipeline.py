"""Oracle side of the parity tests: the FP64 ratio-filter path for chosen templates.

Calls only oracle/ and workload/.  Data are the complex64-rounded spectrum the GPU consumes.
"""
import numpy as np

from oracle import matched, ratio, triggers, waveform as wf


def data32(data):
    return data.dtilde.astype(np.complex64).astype(np.complex128)


class OracleRun:
    def __init__(self, cfg, bank, data, n=None):
        self.cfg = cfg
        self.bank = bank
        self.n = cfg.n if n is None else n
        self.df = cfg.fs / self.n
        self.d = data32(data)
        self.psd = data.psd
        self._q = {}
        self._design = {}

    def q_ref(self, r):
        if r not in self._q:
            h_r = wf.template(self.cfg.fs, self.n, self.cfg.f_low, self.bank.ref_params()[r], self.cfg.pn_flags)
            self._q[r] = matched.filter_unnormalised(self.d, h_r, self.psd, self.df, self.n)
        return self._q[r]

    def design(self, j, K, with_match=True):
        key = (int(j), int(K), bool(with_match))
        if key not in self._design:
            r = int(self.bank.ref_of_tmpl[j])
            self._design[key] = ratio.design(self.cfg.fs, self.n, self.cfg.f_low, self.bank.params()[j],
                                             self.bank.ref_params()[r], self.psd, K, self.cfg.tukey_alpha,
                                             self.cfg.pn_flags, with_match=with_match)
        return self._design[key]

    def snr(self, j, out):
        r = int(self.bank.ref_of_tmpl[j])
        return ratio.snr_series(self.q_ref(r), out["taps"], out["lag"], out["sigma_eff"])

    def snr_at(self, j, out, t):
        r = int(self.bank.ref_of_tmpl[j])
        return ratio.ratio_fir_at(self.q_ref(r), out["taps"], out["lag"], t) / out["sigma_eff"]

    def triggers(self, z, tol):
        return triggers.window_triggers(z, self.cfg.window, self.cfg.threshold, tol=tol)

    def findchirp(self, j):
        h = wf.template(self.cfg.fs, self.n, self.cfg.f_low, self.bank.params()[j], self.cfg.pn_flags)
        return matched.findchirp(self.d, h, self.psd, self.df, self.n)

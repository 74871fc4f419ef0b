"""Writes tests/golden/c1_oracle.json from the FP64 oracle alone (no CUDA code).

C1 workload: 16 s at 1024 Hz of coloured noise, 64 TaylorF2 templates against one
reference at (1.4, 1.4) Msun, K = 64 Tukey(0.1) taps, window 102 samples, |z|^2 > 25.
Recorded per template: lag, sigma_eff, tap match and the ratio-path triggers; for the
injected template (slot 1) also its FINDCHIRP triggers.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workload  # noqa: E402
from oracle import matched, ratio, triggers, waveform as wf  # noqa: E402


def c1_oracle():
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg)
    d32 = data.dtilde.astype(np.complex64).astype(np.complex128)   # the GPU consumes complex64
    df = cfg.fs / cfg.n
    ref = bank.ref_params()[0]
    h_r = wf.template(cfg.fs, cfg.n, cfg.f_low, ref)
    q_r = matched.filter_unnormalised(d32, h_r, data.psd, df, cfg.n)
    rows = []
    for j, p in enumerate(bank.params()):
        out = ratio.design(cfg.fs, cfg.n, cfg.f_low, p, ref, data.psd, cfg.k, cfg.tukey_alpha)
        z = ratio.snr_series(q_r, out["taps"], out["lag"], out["sigma_eff"])
        trig = triggers.window_triggers(z, cfg.window, cfg.threshold)
        rows.append({"j": j, "lag": out["lag"], "sigma_eff": out["sigma_eff"], "match": out["match"],
                     "triggers": [[t["w"], t["t"], t["p"]] for t in trig]})
    m0, snr, phi, slot = data.injections[0]
    h_j = wf.template(cfg.fs, cfg.n, cfg.f_low, bank.params()[slot])
    zf = matched.findchirp(d32, h_j, data.psd, df, cfg.n)
    ftrig = triggers.window_triggers(zf, cfg.window, cfg.threshold)
    return {"config": cfg.name, "injection": {"sample": m0, "snr": snr, "phase": phi, "slot": slot},
            "templates": rows, "findchirp_slot": [[t["w"], t["t"], t["p"]] for t in ftrig]}


if __name__ == "__main__":
    res = c1_oracle()
    with open(os.path.join(HERE, "c1_oracle.json"), "w") as fh:
        json.dump(res, fh, indent=1)
    print("wrote", os.path.join(HERE, "c1_oracle.json"))

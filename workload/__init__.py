"""Seeded synthetic workloads for the ratio-filter matched filter.

This package produces the *inputs* of the method and nothing else: the PSD samples,
the coloured-noise data spectrum with injected chirps, the template-bank parameters,
the reference parameters and the template->reference association.  Both the FP64
oracle (tests only) and the CUDA path consume these arrays; neither side imports the
other, and this package holds none of the method's arithmetic (no matched filter, no
ratio, no taps, no FIR, no triggers).

The injected signals need a waveform, so `_inject` evaluates a TaylorF2 chirp of its
own.  It is data synthesis: the oracle and the kernels each evaluate template phases
with their own code, which is what the injection-recovery tests compare against.
"""
from .configs import CONFIGS, Config, get_config, small_config  # noqa: F401
from .generate import (  # noqa: F401
    Bank, Data, T_SUN, chirp_mass, make_bank, make_data, make_workload, psd_analytic,
    band_low_index, make_training_bank, dense_bank,
)

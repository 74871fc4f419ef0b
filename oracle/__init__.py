"""FP64 CPU oracle for Ratio-Filter Dechirping (arXiv 2601.18835).

TEST INFRASTRUCTURE.  Only the test suite, the package smoke check and the CPU-baseline
leg of the benchmark import this package; the library's product path never does, and it
fails loudly when its CUDA extension is missing.  The oracle shares no code with the CUDA
path: the two meet only in the seeded inputs produced by the `workload` package.

Everything is plain numpy in float64 / complex128, written to be checked against the paper
by eye.  Each function cites the passage it follows:

  fft.py        hand-written iterative radix-2 FFT (the FFT of Eq. 1)
  waveform.py   TaylorF2 templates h(f) = f^(-7/6) exp(-i Psi(f)) (the template of Eq. 1)
  matched.py    FINDCHIRP matched filter, Eq. 1; optimal SNR normalisation
  ratio.py      ratio R = h / h_ref (Eq. 2), taps from the inverse transform of conj(R)
                (Eq. 3 and Sec. V), Tukey window and placement, the direct circular FIR
                (Eq. 3), sigma_eff by Parseval (Eqs. 5-6), tap match, K-bucket choice
  triggers.py   |z|^2 threshold crossings and per-window maxima (Table II's peak find and
                trigger accumulation)

Parity status: every function here is pinned by the CPU tests (brute-force DFT, Parseval,
closed forms, library special cases, injection recovery, the K = N identity of Eq. 3).
"""
from . import fft, waveform, matched, ratio, triggers  # noqa: F401

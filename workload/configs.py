"""The five workload configurations (sizes, mass ranges, seeds) and small test grids.

C1..C5 follow the workload table of the build plan: a 16 s / 1024 Hz parity case,
the offline-shaped 256 s / 2048 Hz bank, the bucketed spin-orbit bank, the tidal
(learned-tap) bank and the long subsolar-mass bank.  Seeds are fixed per config:
bank 1000+c, noise 2000+c, injections 3000+c.
"""
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

PN_SO = 1      # aligned-spin 1.5PN spin-orbit term
PN_TIDAL = 2   # 5PN tidal term


@dataclass(frozen=True)
class Config:
    name: str
    index: int
    fs: float
    n: int
    f_low: float
    n_tmpl: int
    n_ref: int
    k: int                      # fixed tap count (0 = bucketed)
    m_range: Tuple[float, float]
    chi_range: Optional[Tuple[float, float]] = None
    lambda_range: Optional[Tuple[float, float]] = None
    pn_flags: int = 0
    n_inj: int = 8
    inj_snr: Tuple[float, float] = (8.0, 20.0)
    window: int = 205           # samples per trigger window (round(0.1 s * fs))
    threshold: float = 25.0     # |z|^2 threshold (strict >)
    k_buckets: Tuple[int, ...] = ()
    tukey_alpha: float = 0.1
    # C1 special slots: slot 0 = reference, slot 1 = reference with m1 + 0.001
    c1_slots: bool = False
    seeds: Tuple[int, int, int] = field(default=(0, 0, 0))

    @property
    def duration(self) -> float:
        return self.n / self.fs

    @property
    def k_max(self) -> int:
        return max(self.k_buckets) if self.k_buckets else self.k


def _seeds(c):
    return (1000 + c, 2000 + c, 3000 + c)


CONFIGS = {
    1: Config("c1_plain_16s_1024hz", 1, fs=1024.0, n=16384, f_low=30.0, n_tmpl=64, n_ref=1,
              k=64, m_range=(1.2, 1.6), n_inj=1, inj_snr=(12.0, 12.0), window=102,
              c1_slots=True, seeds=_seeds(1)),
    2: Config("c2_offline_256s_2048hz", 2, fs=2048.0, n=524288, f_low=20.0, n_tmpl=4096,
              n_ref=16, k=128, m_range=(1.0, 3.0), seeds=_seeds(2)),
    3: Config("c3_bucketed_spin_orbit", 3, fs=2048.0, n=524288, f_low=20.0, n_tmpl=100000,
              n_ref=64, k=0, m_range=(1.0, 20.0), chi_range=(-0.5, 0.5), pn_flags=PN_SO,
              k_buckets=(32, 64, 128, 256, 512), seeds=_seeds(3)),
    4: Config("c4_learned_taps_tidal", 4, fs=2048.0, n=524288, f_low=20.0, n_tmpl=20000,
              n_ref=16, k=128, m_range=(1.0, 2.5), chi_range=(-0.05, 0.05),
              lambda_range=(0.0, 2000.0), pn_flags=PN_TIDAL, seeds=_seeds(4)),
    5: Config("c5_subsolar_512s_2048hz", 5, fs=2048.0, n=1048576, f_low=45.0, n_tmpl=200000,
              n_ref=256, k=512, m_range=(0.2, 1.0), seeds=_seeds(5)),
}


def get_config(c: int) -> Config:
    return CONFIGS[c]


def small_config(base: int = 2, **kw) -> Config:
    """A reduced copy of a config for tests (same physics, smaller n / bank)."""
    return replace(CONFIGS[base], **kw)

"""Index model of the block-FFT kernel's 2048-point transform (rf_fft.cu: group_fft,
build_twiddles, the swizzled rows), replayed in numpy and checked against a direct DFT.

The model follows the kernel's schedule step by step: thread t of a 128-thread group holds
elements t + 128 r; pass 1 (radix 8, two butterflies per thread) writes position 8 j + r of
tile A; pass 2 (radix 16, ns = 8, twiddle row t mod 8) reads A[t + 128 r] and writes
B[16 (t - k) + k + 8 r]; pass 3 (radix 16, ns = 128, twiddle row 8 + t) reads B[t + 128 r]
and leaves element t + 128 r in the thread.  Tiles are padded by one element per 16
(position i at i + i // 16), and twiddle rows use the XOR-swizzled layout (value r of row i
at 16 i + 2 ((r // 2) ^ (i mod 8)) + r mod 2).  A mistake in any of these index rules makes
the transform wrong.
"""
import numpy as np
import pytest

M, GT = 2048, 128


def tpos(i):
    return i + (i >> 4)


def swz(i, c):
    return 16 * i + 2 * (c ^ (i & 7))


def dft(v, inv):
    R = len(v)
    sign = 1 if inv else -1
    k = np.arange(R)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / R) @ v


def stage_table():
    """The stage twiddles of length 2048 (radix 8 then 16, 16): pass p after ns holds
    w_(ns R)^(r k) at base_p + (r - 1) ns + k."""
    out = np.zeros(M, dtype=np.complex128)
    e, ns = 0, 1
    for R in (8, 16, 16):
        for r in range(1, R):
            for k in range(ns):
                out[e] = np.exp(2j * np.pi * r * k / (ns * R))
                e += 1
        ns *= R
    assert e == M - 1
    return out


def twiddle_rows(stage):
    """build_twiddles: rows k < 8 (pass 2) and 8 + t (pass 3), value 0 = 1, swizzled."""
    tw = np.zeros((8 + GT) * 16, dtype=np.complex128)
    for i in range(8 + GT):
        for r in range(16):
            w = 1.0 + 0j
            if r > 0:
                w = stage[7 + (r - 1) * 8 + i] if i < 8 else stage[127 + (r - 1) * GT + (i - 8)]
            tw[swz(i, r >> 1) + (r & 1)] = w
    return tw


def load_row16(tw, i):
    return np.array([tw[swz(i, c) + h] for c in range(8) for h in (0, 1)])


def group_fft(V, tw, inv):
    """V[t][r] = element t + 128 r on entry and exit."""
    A = np.full(M + M // 16 + 2, np.nan + 0j)
    B = np.full(M + M // 16 + 2, np.nan + 0j)
    for t in range(GT):
        a = dft(np.array([V[t][2 * r] for r in range(8)]), inv)
        b = dft(np.array([V[t][2 * r + 1] for r in range(8)]), inv)
        for r in range(8):
            A[tpos(8 * t + r)] = a[r]
            A[tpos(8 * (t + GT) + r)] = b[r]
    for t in range(GT):
        k = t & 7
        v = np.array([A[tpos(t + GT * r)] for r in range(16)])
        w = load_row16(tw, k)
        v[1:] *= w[1:] if inv else np.conj(w[1:])
        v = dft(v, inv)
        idx = ((t - k) << 4) + k
        for r in range(16):
            B[tpos(idx + 8 * r)] = v[r]
    out = np.zeros((GT, 16), dtype=np.complex128)
    for t in range(GT):
        v = np.array([B[tpos(t + GT * r)] for r in range(16)])
        w = load_row16(tw, 8 + t)
        v[1:] *= w[1:] if inv else np.conj(w[1:])
        out[t] = dft(v, inv)
    return out


@pytest.mark.parametrize("inv", [False, True])
def test_group_fft_index_scheme_is_a_dft(inv):
    rng = np.random.default_rng(11)
    x = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    V = np.array([[x[t + GT * r] for r in range(16)] for t in range(GT)])
    got = group_fft(V, twiddle_rows(stage_table()), inv)
    y = np.array([got[i % GT][i // GT] for i in range(M)])
    ref = np.fft.ifft(x) * M if inv else np.fft.fft(x)
    assert np.max(np.abs(y - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_swizzled_rows_are_conflict_free():
    """Eight consecutive rows read chunk c: the 16-byte units land in eight different bank
    groups (unit mod 8), for every c."""
    for i0 in range(0, 136, 8):
        for c in range(8):
            groups = {(swz(i, c) // 2) % 8 for i in range(i0, i0 + 8)}
            assert len(groups) == 8

"""Index model of the two-pass (four-step) Stockham FFT (fft.cu: k_fft_cols, k_fft_rows,
block_fft and its passes), replayed in numpy against numpy's FFT.

The model follows the kernels' rules: n = N1 N2 with N1 = 2^ceil(log2 n / 2); the column
kernel takes C adjacent columns, the row kernel C rows (C = max(c_min, 2^log_min_el / L) capped
by the other dimension); the shared tile holds column c, element i at c LP + i + i // 16,
LP = L + L / 16 + 2; the first radix pass (radix 2, 4, 8 or 16) reads global memory, middle
radix-16 passes run in the tile with stage twiddles w_(ns R)^(r k) at base + (r - 1) ns + k,
and the last pass writes global memory, the column kernel multiplying by
w_n^(n2 k1) = hi[m >> s] lo[m mod 2^s].  A mistake in the pass, twiddle or mapping rules makes
the transform wrong (a tile position written twice or read unwritten shows as a wrong or NaN
result); the padding itself only decides bank conflicts, which the last test checks.
"""
import numpy as np
import pytest


def tile_ld(L):
    return L + L // 16 + 2


def pos(c, i, LP):
    return c * LP + i + (i >> 4)


def dft(v, inv):
    R = len(v)
    k = np.arange(R)
    return np.exp((1 if inv else -1) * 2j * np.pi * np.outer(k, k) / R) @ v


def stage_tw(logL):
    L = 1 << logL
    out, e, ns = np.zeros(L, dtype=np.complex128), 0, 1
    first = logL & 3
    for R in ([1 << first] if first else []) + [16] * (logL // 4):
        for r in range(1, R):
            for k in range(ns):
                out[e] = np.exp(2j * np.pi * r * k / (ns * R))
                e += 1
        ns *= R
    assert e == L - 1
    return out


def block_fft(logL, logC, stw, gin, in_ld, in_cs, gout, out_ld, inv, outer=None):
    """One block: C transforms of length L from gin (element (c, i) at i in_ld + c in_cs) to
    gout (element (c, k) at k out_ld + c); outer = (c0, s, lo, hi) for the column kernel."""
    L, C = 1 << logL, 1 << logC
    LP = tile_ld(L)
    S = np.full(C * LP, np.nan + 0j)
    first = logL & 3
    R0 = (1 << first) if first else 16
    lr = L // R0
    for c in range(C):                                   # first pass: global -> tile, ns = 1
        for j in range(lr):
            v = dft(np.array([gin[(j + r * lr) * in_ld + c * in_cs] for r in range(R0)]), inv)
            for r in range(R0):
                S[pos(c, j * R0 + r, LP)] = v[r]
    off, ns = R0 - 1, R0
    npass = (1 if first else 0) + logL // 4
    for _ in range(1, npass - 1):                        # middle passes: in place, radix 16
        lr = L // 16
        vals = []
        for c in range(C):
            for j in range(lr):
                k = j & (ns - 1)
                v = np.array([S[pos(c, j + r * lr, LP)] for r in range(16)])
                w = stw[off + np.arange(15) * ns + k]
                v[1:] *= w if inv else np.conj(w)
                vals.append((c, j, k, dft(v, inv)))
        for c, j, k, v in vals:
            idx = ((j - k) << 4) + k
            for r in range(16):
                S[pos(c, idx + r * ns, LP)] = v[r]
        off, ns = off + 15 * ns, ns * 16
    lr = L // 16                                         # last pass: tile -> global, k = j
    for c in range(C):
        for j in range(lr):
            v = np.array([S[pos(c, j + r * lr, LP)] for r in range(16)])
            w = stw[off + np.arange(15) * lr + j]
            v[1:] *= w if inv else np.conj(w)
            v = dft(v, inv)
            for r in range(16):
                k = j + r * lr
                o = v[r]
                if outer is not None:
                    c0, s, lo, hi = outer
                    m = (c0 + c) * k
                    wo = hi[m >> s] * lo[m & ((1 << s) - 1)]
                    o = o * (wo if inv else np.conj(wo))
                gout[k * out_ld + c] = o


def two_pass(x, inv, fp32):
    n = len(x)
    log2n = n.bit_length() - 1
    log_min_el, log_min_c = (13, 3) if fp32 else (12, 2)
    logN1 = (log2n + 1) // 2
    logN2 = log2n - logN1
    N1, N2 = 1 << logN1, 1 << logN2

    def pick(logL, log_other):
        return min(max(log_min_c, log_min_el - logL), log_other)

    logCA, logCB = pick(logN1, logN2), pick(logN2, logN1)
    s = (log2n + 1) // 2
    lo = np.exp(2j * np.pi * np.arange(1 << s) / n)
    hi = np.exp(2j * np.pi * np.arange(n >> s) / (n >> s))
    y = np.zeros(n, dtype=np.complex128)
    out = np.zeros(n, dtype=np.complex128)
    stA, stB = stage_tw(logN1), stage_tw(logN2)
    for bx in range(N2 >> logCA):
        c0 = bx * (1 << logCA)
        tmp = np.zeros(n, dtype=np.complex128)
        block_fft(logN1, logCA, stA, x[c0:], N2, 1, tmp, N2, inv, (c0, s, lo, hi))
        for k1 in range(N1):
            y[k1 * N2 + c0: k1 * N2 + c0 + (1 << logCA)] = tmp[k1 * N2: k1 * N2 + (1 << logCA)]
    for bx in range(N1 >> logCB):
        r0 = bx * (1 << logCB)
        tmp = np.zeros(n, dtype=np.complex128)
        block_fft(logN2, logCB, stB, y[r0 * N2:], 1, N2, tmp, N1, inv)
        for k2 in range(N2):
            out[k2 * N1 + r0: k2 * N1 + r0 + (1 << logCB)] = tmp[k2 * N1: k2 * N1 + (1 << logCB)]
    return out


@pytest.mark.parametrize("log2n,fp32", [(12, True), (12, False), (13, True), (13, False)])
@pytest.mark.parametrize("inv", [False, True])
def test_two_pass_index_scheme_is_a_dft(log2n, fp32, inv):
    n = 1 << log2n
    rng = np.random.default_rng(log2n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = two_pass(x, inv, fp32)
    ref = np.fft.ifft(x) * n if inv else np.fft.fft(x)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.sqrt(np.mean(np.abs(ref) ** 2))


def test_two_pass_with_a_middle_pass():
    """n = 2^17: transforms of length 512 (radix 2, 16, 16: one middle pass in the tile)."""
    n = 1 << 17
    rng = np.random.default_rng(17)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = two_pass(x, True, True)
    ref = np.fft.ifft(x) * n
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.sqrt(np.mean(np.abs(ref) ** 2))


def _slots(addrs):
    """Shared-memory 8-byte slots of one half-warp's float2 accesses (16 slots per 128 B)."""
    return [a % 16 for a in addrs]


@pytest.mark.parametrize("logL", [9, 10, 11])
def test_padding_keeps_the_radix16_scatter_conflict_free(logL):
    """The first pass of radix 16 writes j * 16 + r: one pad per 16 elements spreads a
    half-warp's 16 writes over 16 different slots, whether the lanes run along j (one column)
    or along 8 adjacent columns and two j (the column kernel's mapping); the last pass's reads
    j + r L/16 along 8 columns conflict at most 2-way."""
    L = 1 << logL
    LP = tile_ld(L)
    for r in range(16):
        for j0 in range(0, L // 16, 16):                 # lanes along j
            assert len(set(_slots([pos(0, (j0 + l) * 16 + r, LP) for l in range(16)]))) == 16
        for j0 in range(0, L // 16, 2):                  # lanes along 8 columns x 2 j
            assert len(set(_slots([pos(c, (j0 + jj) * 16 + r, LP) for jj in (0, 1) for c in range(8)]))) == 16
        for j0 in range(0, L // 16, 2):
            sl = _slots([pos(c, (j0 + jj) + r * (L // 16), LP) for jj in (0, 1) for c in range(8)])
            assert max(sl.count(x) for x in set(sl)) <= 2

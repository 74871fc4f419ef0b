"""Tap banks on disk (rfd_taps_key, rfd_make_taps_cached).

CPU: the key is the SHA-256 (Python's hashlib, an implementation independent of the library's)
of the serialisation include/rfd.h documents, for both tap policies and for message lengths that
cover every SHA-256 padding case; one ulp of the PSD, the Tukey parameter or one template's K
changes it.  GPU: a miss extracts and stores the bank, a hit reads back exactly what
rfd_make_taps writes; a changed PSD, a truncated file and a request for the match that the file
lacks are misses that replace the file."""
import hashlib
import os
import re
import struct

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rfd():
    from paper_2601_18835_gb300 import build
    build.build()
    import paper_2601_18835_gb300 as m
    return m


def version():
    text = open(os.path.join(ROOT, "include", "rfd.h")).read()
    return int(re.search(r"#define RFD_VERSION (\d+)", text).group(1))


def serialise(g, psd, refs, tmpl, ref_of, k, k_stride, alpha, buckets=None, energy_frac=0.999):
    mode = 0 if k is not None else 1
    nb = 0 if mode == 0 else len(buckets)
    b = b"librfd-taps\x00" + struct.pack("<ii", version(), mode)
    b += struct.pack("<dqdi", g.fs, g.n, g.f_low, g.pn_flags)
    b += struct.pack("<iii", len(refs), len(tmpl), k_stride)
    b += struct.pack("<ddi", alpha, energy_frac if mode else 0.0, nb)
    b += np.asarray(refs, "<f8").tobytes() + np.asarray(tmpl, "<f8").tobytes() + np.asarray(ref_of, "<i4").tobytes()
    b += np.asarray(k if mode == 0 else buckets, "<i4").tobytes()
    b += np.asarray(psd, "<f8").tobytes()
    return b


def bank(rng, n_ref, n_tmpl):
    refs = rng.uniform(1.0, 3.0, size=(n_ref, 5))
    tmpl = rng.uniform(1.0, 3.0, size=(n_tmpl, 5))
    ref_of = rng.integers(0, n_ref, size=n_tmpl).astype(np.int32)
    return refs, tmpl, ref_of


def test_key_is_sha256_of_the_documented_serialisation(rfd):
    rng = np.random.default_rng(5)
    g = rfd.grid(2048.0, 4096, 20.0, 1)
    psd = rng.uniform(1e-47, 1e-45, size=4096 // 2 + 1)
    lengths = set()
    for n_ref in (1, 2):
        for n_tmpl in range(0, 5):
            refs, tmpl, ref_of = bank(rng, n_ref, n_tmpl)
            k = rng.integers(1, 128, size=n_tmpl).astype(np.int32)
            msg = serialise(g, psd, refs, tmpl, ref_of, k, 128, 0.1)
            assert rfd.taps_key(g, psd, refs, tmpl, ref_of, k, 128, 0.1) == hashlib.sha256(msg).digest()
            lengths.add(len(msg) % 64)
            for nb in range(1, 17):                      # 4-byte steps through the last block
                buckets = np.arange(1, nb + 1, dtype=np.int32) * 8
                msg = serialise(g, psd, refs, tmpl, ref_of, None, 128, 0.1, buckets, 0.99)
                got = rfd.taps_key(g, psd, refs, tmpl, ref_of, None, 128, 0.1, buckets=buckets, energy_frac=0.99)
                assert got == hashlib.sha256(msg).digest()
                lengths.add(len(msg) % 64)
    # every message length here is a multiple of 4; the padding's cases: the 0x80 byte and the
    # 8-byte length fit the last block (up to 55 bytes used), or need an extra block (56 and up)
    assert {0, 52, 56, 60} <= lengths


def test_key_follows_every_input(rfd):
    rng = np.random.default_rng(6)
    g = rfd.grid(1024.0, 2048, 30.0)
    psd = rng.uniform(1e-47, 1e-45, size=1025)
    refs, tmpl, ref_of = bank(rng, 2, 6)
    k = np.full(6, 64, dtype=np.int32)
    base = rfd.taps_key(g, psd, refs, tmpl, ref_of, k, 64, 0.1)
    assert rfd.taps_key(g, psd.copy(), refs.copy(), tmpl.copy(), ref_of.copy(), k.copy(), 64, 0.1) == base
    p2 = psd.copy()
    p2[100] = np.nextafter(p2[100], np.inf)
    k2 = k.copy()
    k2[3] = 63
    t2 = tmpl.copy()
    t2[2, 4] = 1e-300
    for other in (rfd.taps_key(g, p2, refs, tmpl, ref_of, k, 64, 0.1),
                  rfd.taps_key(g, psd, refs, tmpl, ref_of, k2, 64, 0.1),
                  rfd.taps_key(g, psd, refs, t2, ref_of, k, 64, 0.1),
                  rfd.taps_key(g, psd, refs, tmpl, ref_of, k, 64, np.nextafter(0.1, 1.0)),
                  rfd.taps_key(g, psd, refs, tmpl, ref_of, k, 128, 0.1),
                  rfd.taps_key(rfd.grid(1024.0, 2048, 30.0, 2), psd, refs, tmpl, ref_of, k, 64, 0.1)):
        assert other != base


def test_key_rejects_a_bad_grid(rfd):
    g = rfd.grid(1024.0, 1000, 30.0)                     # not a power of two
    with pytest.raises(rfd.RfdError):
        rfd.taps_key(g, np.ones(501), np.ones((1, 5)), np.ones((1, 5)), [0], [8], 8, 0.1)


@pytest.mark.gpu
def test_cache_miss_then_hit(rfd, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import workload
    from tests.gpu_pipeline import GpuRun

    cfg = workload.small_config(1, n_tmpl=40, n_ref=2, c1_slots=False)
    bk, data = workload.make_workload(cfg)
    gpu = GpuRun(cfg, bk, data)
    K = np.array([16, 33, 64, 64, 7] * 8, dtype=np.int32)
    J = len(K)

    def outputs(match):
        return (torch.zeros((J, 64), dtype=torch.complex64, device="cuda"),
                torch.zeros(J, dtype=torch.int32, device="cuda"), torch.zeros(J, dtype=torch.float64, device="cuda"),
                torch.zeros(J, dtype=torch.float64, device="cuda") if match else None,
                torch.zeros(J, dtype=torch.int32, device="cuda"))

    def cached(psd, match):
        taps, lag, sig, mat, kk = outputs(match)
        hit = rfd.make_taps_cached(str(tmp_path / "bank"), gpu.ctx, gpu.grid, psd, bk.ref_params(), bk.params(),
                                   bk.ref_of_tmpl, K, 64, cfg.tukey_alpha, taps, lag, sig, mat, k_out=kk)
        torch.cuda.synchronize()
        return hit, [x.cpu().numpy().tobytes() if x is not None else None for x in (taps, lag, sig, mat, kk)]

    ref = gpu.make_taps(K, k_stride=64, match=True)
    want = [ref[n].cpu().numpy().tobytes() for n in ("taps", "lag", "sigma", "match")]
    hit, got = cached(gpu.psd, match=False)
    assert not hit and got[:3] == want[:3] and np.array_equal(np.frombuffer(got[4], np.int32), K)
    key = rfd.taps_key(gpu.grid, data.psd, bk.ref_params(), bk.params(), bk.ref_of_tmpl, K, 64, cfg.tukey_alpha)
    path = tmp_path / "bank" / (key.hex() + ".rfdtaps")
    assert path.exists() and sorted(os.listdir(tmp_path / "bank")) == [path.name]
    hit, got = cached(gpu.psd, match=False)
    assert hit and got[:3] == want[:3] and np.array_equal(np.frombuffer(got[4], np.int32), K)
    # the file lacks the match: a miss that stores it; then a hit with it
    hit, got = cached(gpu.psd, match=True)
    assert not hit and got[:4] == want
    hit, got = cached(gpu.psd, match=True)
    assert hit and got[:4] == want
    # a truncated file is a miss and is replaced
    size = path.stat().st_size
    with open(path, "r+b") as fh:
        fh.truncate(size - 8)
    hit, got = cached(gpu.psd, match=True)
    assert not hit and got[:4] == want and path.stat().st_size == size
    # one ulp of the PSD is another bank
    psd2 = data.psd.copy()
    psd2[500] = np.nextafter(psd2[500], np.inf)
    hit, _ = cached(torch.from_numpy(psd2).cuda(), match=False)
    assert not hit and len(os.listdir(tmp_path / "bank")) == 2

"""The C ABI from a plain C99 program (tests/abi_c/pipeline.c): include/rfd.h compiles under
-std=c99 -pedantic -Werror, the library links without C++ or Python, its host-only entry points
answer as documented (CPU), and the whole path driven from C -- reference templates, the
reference matched filter (Eq. 1), taps (Sec. V), the ratio filter (Eq. 3) and the trigger
reduction -- gives the same bytes as the Python binding on the same inputs, and the oracle's
triggers (GPU)."""
import glob
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "abi_c", "pipeline.c")


def cuda_home():
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nv)))


def cuda_libdir(home):
    for d in [os.path.join(home, "lib64")] + sorted(glob.glob(os.path.join(home, "targets", "*", "lib"))):
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    pytest.skip("libcudart.so not found under %s" % home)


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    from paper_2601_18835_gb300 import build
    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    home = cuda_home()
    libdir = cuda_libdir(home)
    out = str(tmp_path_factory.mktemp("abi_c") / "pipeline")
    cmd = [cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-O1", "-I", os.path.join(ROOT, "include"),
           "-isystem", os.path.join(home, "include"), SRC, "-o", out, lib, "-L", libdir, "-lcudart",
           "-Wl,-rpath," + os.path.dirname(lib) + ":" + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def test_header_is_c99_and_host_calls_answer(exe):
    header = open(os.path.join(ROOT, "include", "rfd.h")).read()
    r = subprocess.run([exe, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    assert int(out["version"]) == int(re.search(r"#define RFD_VERSION (\d+)", header).group(1))
    assert out["qref_ld"].split() == ["524416", "1088"]
    assert out["status"] == "output capacity exceeded|device wait timed out"
    # the defaults the header states: tile_nt = {128, 64, 32}, mix_k = 1, grid_ctas = 0,
    # long_k = 64, fft_k = 4096, out_len = 0, fft_rem = 0, debug_flags = 0
    assert [int(x) for x in out["options"].split()] == [128, 64, 32, 1, 0, 64, 4096, 0, 0, 0]
    # record sizes the header states (24- and 20-byte records), and the grid / parameter structs
    assert [int(x) for x in out["sizes"].split()] == [24, 20, 32, 40]
    st, ctx = out["ctx_create(-1)"].split()
    assert int(st) < 0 and ctx == "null"


def write_input(path, cfg, bank, data, K, prec, halo):
    n = cfg.n
    with open(path, "wb") as f:
        np.array([n, bank.n_ref, bank.n_tmpl, K, cfg.window, prec, cfg.pn_flags, halo], dtype="<i8").tofile(f)
        np.array([cfg.fs, cfg.f_low, cfg.threshold, cfg.tukey_alpha], dtype="<f8").tofile(f)
        np.ascontiguousarray(bank.ref_params(), dtype="<f8").tofile(f)
        np.ascontiguousarray(bank.params(), dtype="<f8").tofile(f)
        np.ascontiguousarray(bank.ref_of_tmpl, dtype="<i4").tofile(f)
        np.ascontiguousarray(data.psd, dtype="<f8").tofile(f)
        np.ascontiguousarray(data.dtilde.astype(np.complex64)).view("<f4").tofile(f)


def read_output(path, n_tmpl):
    import paper_2601_18835_gb300 as rfd
    raw = open(path, "rb").read()
    n_cand, n_trig = np.frombuffer(raw[:16], dtype="<i8")
    off = 16
    trig = np.frombuffer(raw[off:off + 20 * n_trig], dtype=rfd.TRIGGER_DTYPE)
    off += 20 * n_trig
    lag = np.frombuffer(raw[off:off + 4 * n_tmpl], dtype="<i4")
    off += 4 * n_tmpl
    sigma = np.frombuffer(raw[off:off + 8 * n_tmpl], dtype="<f8")
    assert off + 8 * n_tmpl == len(raw)
    return int(n_cand), trig, lag, sigma


@pytest.mark.gpu
@pytest.mark.parametrize("prec_name", ["fp32", "fp16x3"])
def test_whole_path_from_c(exe, tmp_path, prec_name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_18835_gb300 as rfd
    import workload
    from tests.gpu_pipeline import GpuRun
    from tests.oracle_pipeline import OracleRun
    from tests.test_gpu_parity import EPS, TOL_FP32, TOL_TC, amb_cap, compare_triggers, n_oracle, snr_errors

    prec = {"fp32": rfd.PREC_FP32, "fp16x3": rfd.PREC_FP16X3}[prec_name]
    cfg = workload.get_config(1)
    bank, data = workload.make_workload(cfg)
    halo = cfg.k - 1
    inp, outp = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    write_input(inp, cfg, bank, data, cfg.k, prec, halo)
    r = subprocess.run([exe, "run", inp, outp], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    n_cand, trig, lag, sigma = read_output(outp, bank.n_tmpl)

    # the same calls through the Python binding: the same bytes
    gpu = GpuRun(cfg, bank, data)
    t = gpu.make_taps(cfg.k, match=False)
    assert np.array_equal(lag, t["lag"].cpu().numpy())
    assert np.array_equal(sigma, t["sigma"].cpu().numpy())
    q, e, _ = gpu.filter_reference(halo, prec)
    trig_py, n_cand_py = gpu.ratio_filter(t, q, e, prec, halo)
    assert n_cand == n_cand_py and trig.tobytes() == trig_py.tobytes()

    # and the oracle's triggers
    ora = OracleRun(cfg, bank, data)
    sets = {j: ora.triggers(ora.snr(j, ora.design(j, cfg.k, with_match=False)), EPS[prec])
            for j in range(bank.n_tmpl)}
    tol = TOL_FP32 if prec == rfd.PREC_FP32 else TOL_TC
    assert compare_triggers(trig, sets, tol, range(bank.n_tmpl), cfg.window) <= amb_cap(
        n_oracle(sets, range(bank.n_tmpl)))
    assert snr_errors(trig, sets, range(bank.n_tmpl)) < EPS[prec]

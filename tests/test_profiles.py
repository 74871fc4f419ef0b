"""The committed ncu summaries describe the committed sources: every summary marked current in
profiles/README.md and every DRAM figure in profiles/traffic.json carries the source hash that
bench.py computes for its kernel now, and every bench.py command a summary gives uses options
bench.py has."""
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")

# summary file / traffic key -> the kernel source file its hash covers
SUMMARY_SOURCE = {"k_rf_tc_long_c2.md": "rf_tc_long.cu", "k_rf_tc_c2.md": "rf_tc.cu", "k_rf_fft_c2.md": "rf_fft.cu",
                  "k_fir32_c2.md": "fir32.cu", "findchirp_c2.md": "fft.cu"}
TRAFFIC_SOURCE = {"k_rf_tc_long": "rf_tc_long.cu", "k_rf_tc": "rf_tc.cu", "k_rf_fft": "rf_fft.cu",
                  "k_fir32": "fir32.cu"}


@pytest.fixture(scope="module")
def source_hash():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_for_profiles", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    return bench.kernel_source_hash


def test_index_rows_marked_current_match_the_sources(source_hash):
    rows = [line for line in open(os.path.join(PROFILES, "README.md")) if line.startswith("| `")]
    seen = set()
    for row in rows:
        name = re.match(r"\| `([^`]+)`", row).group(1)
        m = re.search(r"current \(`([0-9a-f]{16})`\)", row)
        if m is None:
            continue
        assert name in SUMMARY_SOURCE, name
        assert m.group(1) == source_hash(SUMMARY_SOURCE[name]), name
        # the summary itself names the same hash
        assert m.group(1) in open(os.path.join(PROFILES, name)).read(), name
        seen.add(name)
    assert seen == set(SUMMARY_SOURCE)


def test_traffic_figures_match_the_sources(source_hash):
    with open(os.path.join(PROFILES, "traffic.json")) as fh:
        rec = json.load(fh)
    for kernel, src in TRAFFIC_SOURCE.items():
        assert rec[kernel]["source_sha"] == source_hash(src), kernel


def test_summary_commands_use_existing_bench_options():
    bench_src = open(os.path.join(ROOT, "bench.py")).read()
    options = set(re.findall(r'add_argument\("(--[a-z0-9-]+)"', bench_src))
    for name in os.listdir(PROFILES):
        if not name.endswith(".md"):
            continue
        text = open(os.path.join(PROFILES, name)).read().replace("\\\n", " ")
        for cmd in re.findall(r"python bench\.py([^\n`>|&]*)", text):
            for opt in re.findall(r"(--[a-z0-9-]+)", cmd):
                assert opt in options, (name, opt)

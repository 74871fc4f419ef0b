"""C1 end-to-end on the oracle: injection recovery, the 1 % agreement between the ratio path
and FINDCHIRP for a well-matched template, and a regression against the recorded fixture
(tests/golden/c1_oracle.json, written by tests/golden/make_golden.py from the oracle alone)."""
import json
import os

import numpy as np
import pytest

from tests.golden.make_golden import c1_oracle

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def c1():
    return c1_oracle()


def test_injection_recovered_at_its_sample_and_snr(c1):
    m0 = c1["injection"]["sample"]
    slot = c1["injection"]["slot"]
    trig = c1["templates"][slot]["triggers"]
    assert len(trig) == 1
    w, t, p = trig[0]
    assert abs(t - m0) <= 1
    assert 9.0 <= np.sqrt(p) <= 15.0        # SNR 12 +- 3 in this noise realisation


def test_ratio_peak_within_one_percent_of_findchirp(c1):
    slot = c1["injection"]["slot"]
    row = c1["templates"][slot]
    assert row["match"] >= 0.99
    p_ratio = row["triggers"][0][2]
    p_fc = c1["findchirp_slot"][0][2]
    assert abs(np.sqrt(p_ratio) / np.sqrt(p_fc) - 1.0) < 0.01


def test_identity_slot_has_delta_lag(c1):
    assert c1["templates"][0]["lag"] == -32
    assert abs(c1["templates"][0]["match"] - 1.0) < 1e-12


def test_matches_recorded_fixture(c1):
    with open(os.path.join(HERE, "golden", "c1_oracle.json")) as fh:
        rec = json.load(fh)
    assert rec["injection"] == c1["injection"]
    for a, b in zip(rec["templates"], c1["templates"]):
        assert a["lag"] == b["lag"]
        assert abs(a["sigma_eff"] - b["sigma_eff"]) <= 1e-12 * a["sigma_eff"]
        assert abs(a["match"] - b["match"]) <= 1e-12
        assert [x[:2] for x in a["triggers"]] == [x[:2] for x in b["triggers"]]

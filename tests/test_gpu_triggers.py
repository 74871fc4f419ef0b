"""rfd_find_triggers on synthetic candidate lists against a plain per-window maximum.

The merge (Table II's trigger accumulation) must return, per (template, window), the
candidate with the largest key (largest |z|^2, ties to the smallest t), sorted by (j, w),
whatever the order of the list.  The lists here exercise both merge paths: templates with at
most 32 candidates and templates with up to several thousand spread over more windows than
one shared-memory range holds, with exact |z|^2 ties inside windows and duplicated records.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2601_18835_gb300 as rfd  # noqa: E402


def synthetic_candidates(rng, n_tmpl, W):
    recs = []
    for j in range(n_tmpl):
        kind = j % 5
        if kind == 0:
            c, nw = 0, 1
        elif kind == 1:
            c, nw = int(rng.integers(1, 33)), 40
        elif kind == 2:
            c, nw = 32, 8                       # exactly at the warp path's limit, dense windows
        elif kind == 3:
            c, nw = int(rng.integers(33, 400)), 50
        else:
            c, nw = int(rng.integers(1000, 6000)), 9000     # several shared-memory ranges
        w = rng.integers(0, nw, size=c)
        t = w * W + rng.integers(0, W, size=c)
        p = rng.choice(np.float32([25.5, 30.0, 31.25, 100.0]), size=c) + rng.integers(0, 3, size=c).astype(np.float32)
        for i in range(c):
            recs.append((j, int(t[i]), np.float32(p[i])))
            if rng.uniform() < 0.05:           # an identical duplicate of the same record
                recs.append((j, int(t[i]), np.float32(p[i])))
    order = rng.permutation(len(recs))
    return [recs[i] for i in order]


def expected_triggers(recs, W):
    best = {}
    for j, t, p in recs:
        key = (int(np.float32(p).view(np.uint32)) << 32) | (0xFFFFFFFF - t)
        k = (j, t // W)
        if k not in best or key > best[k][0]:
            best[k] = (key, t, p)
    out = []
    for (j, w) in sorted(best):
        key, t, p = best[(j, w)]
        out.append((j, t, p))
    return out


@pytest.mark.parametrize("seed", [1, 2])
def test_merge_equals_per_window_maximum(seed):
    rng = np.random.default_rng(seed)
    W, n_tmpl = 37, 60
    recs = synthetic_candidates(rng, n_tmpl, W)
    cand = np.zeros(len(recs), dtype=rfd.CANDIDATE_DTYPE)
    for i, (j, t, p) in enumerate(recs):
        cand[i]["key"] = (int(np.float32(p).view(np.uint32)) << 32) | (0xFFFFFFFF - t)
        cand[i]["j"] = j
        cand[i]["w"] = t // W
        cand[i]["zr"] = np.float32(np.sqrt(p))    # z identifies the record
        cand[i]["zi"] = np.float32(t)
    ctx = rfd.Context(0)
    cd = torch.from_numpy(cand.view(np.uint8).copy()).cuda()
    cnt = torch.tensor([len(recs)], dtype=torch.int64, device="cuda")
    exp = expected_triggers(recs, W)
    trig = torch.zeros((len(exp) + 16) * 20, dtype=torch.uint8, device="cuda")
    nt = rfd.find_triggers(ctx, n_tmpl, cd, cnt, trig)
    got = rfd.triggers_to_numpy(trig, nt)
    assert nt == len(exp)
    assert [(int(x["j"]), int(x["t"])) for x in got] == [(j, t) for (j, t, _) in exp]
    assert np.array_equal(got["snr2"], np.float32([p for (_, _, p) in exp]))
    assert np.array_equal(got["zi"], got["t"].astype(np.float32))
    ctx.close()

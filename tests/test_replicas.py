"""Multi-GPU path as replicas, on CPU with two gloo ranks (no GPU needed).

bench.py runs one process per GPU; each rank filters its own data segment with the whole
bank (no data-path collective), the job's step time is the maximum over ranks and the rate
counts every rank's templates.  These tests run that host logic with world size 2."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench.dist_env()
        step = [0.010, 0.013][rank]
        m = bench.max_over_ranks(step, got_ws, device="cpu")
        cfg, bank, data = bench.workload_for_rank(1, got_rank, n_tmpl=8)
        out[rank] = (got_ws, got_rank, m, bench.job_rate(got_ws, bank.n_tmpl, cfg.duration, m),
                     float(np.abs(data.dtilde).sum()), tuple(np.round(bank.params()[:, 0], 12)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_own_segments():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        r0, r1 = out[0], out[1]
    assert (r0[0], r0[1], r1[0], r1[1]) == (2, 0, 2, 1)
    assert r0[2] == r1[2] == pytest.approx(0.013)              # the slowest rank sets the step time
    assert r0[3] == pytest.approx(2 * 8 * 16.0 / 0.013)        # both ranks' templates count
    assert r0[4] != r1[4]                                       # each rank has its own noise segment
    assert r0[5] == r1[5]                                       # and the same bank


def test_single_rank_is_plain():
    assert bench.job_rate(1, 4096, 256.0, 0.005) == pytest.approx(4096 * 256.0 / 0.005)
    assert bench.max_over_ranks(0.5, 1, device="cpu") == 0.5

"""The benchmark's multi-rank bookkeeping on CPU (gloo, world size 2).

Under torchrun the job (16 parameter sets per rank) is split across the ranks
by path count; the job's time is the slowest rank's, and the reported rate
counts the units of all ranks.  Checked with two CPU processes: the
max-over-ranks reduction, the whole-job rate, and each rank's share of the
job's flat path list (contiguous, equal, covering it once).  The split call
itself is checked in tests/test_sharding.py and tests/test_gpu_sharding.py.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_seconds = 1.5 + rank          # rank 1 is the slower one
        t_max = bench.max_over_ranks(local_seconds)
        rate = bench.whole_job_rate(1000, world, t_max)
        ws, rk, lr = bench._dist()
        from paper_2302_05170_b300 import sharding
        q.put((rank, t_max, rate, sharding.rank_range(16 * world * 10 ** 6, ws, rk), ws))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, rate, share, ws in out:
        assert ws == 2
        assert t_max == pytest.approx(2.5)
        assert rate == pytest.approx(2 * 1000 / 2.5)
    assert [o[3] for o in out] == [(0, 16 * 10 ** 6), (16 * 10 ** 6, 16 * 10 ** 6)]


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (1, 0, 0)
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0

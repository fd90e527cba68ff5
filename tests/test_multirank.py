"""The benchmark's multi-rank bookkeeping on CPU (gloo, world size 2).

Under torchrun every rank runs its own copy of the workload with its own
Philox key (no collective on the data path); the job's time is the slowest
rank's, and the reported rate counts the units of all ranks.  Checked with
two CPU processes: the max-over-ranks reduction, the whole-job rate and the
per-rank seeds.
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
        q.put((rank, t_max, rate, bench.rank_seed(1, rk), ws))
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
    for rank, t_max, rate, seed, ws in out:
        assert ws == 2
        assert t_max == pytest.approx(2.5)
        assert rate == pytest.approx(2 * 1000 / 2.5)
    assert [o[3] for o in out] == [1, 2]


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (1, 0, 0)
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0

"""One batched 7L call split across ranks: the host side, on CPU.

* rank_range cuts the flat path list into contiguous ranges that cover it exactly once and
  differ in length by at most one path (every path costs the same n_steps evaluations).
* combine_moments merges per-rank (count, mean, variance) in rank order into the batch's
  per-set mean and unbiased variance: against numpy on the concatenated values, with empty
  ranks, single-path ranks and sets split over several ranks.
* Two gloo ranks (separate processes, 127.0.0.1) each run their range -- here through the FP64
  oracle, since the host has no GPU -- gather the partials with one all-gather and combine
  them: every rank gets the same per-set moments, equal to those of the whole batch to
  rounding, and the concatenated per-path values equal the whole batch's bit for bit (the
  normals depend on (set, path within the set, step) only).  The GPU side of the range call
  is checked in tests/test_gpu_sharding.py.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2302_05170_b300 import sharding
from paper_2302_05170_b300 import workloads as W


@pytest.mark.parametrize("total", [0, 1, 5, 1000, 16_000_001])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_rank_range_covers_once(total, world):
    ranges = [sharding.rank_range(total, world, r) for r in range(world)]
    assert ranges[0][0] == 0
    for (a, n), (b, _) in zip(ranges, ranges[1:]):
        assert a + n == b
    assert sum(n for _, n in ranges) == total
    sizes = [n for _, n in ranges]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharding.rank_range(total, world, world)


def _set_moments(values, offsets):
    n_sets = len(offsets) - 1
    c, mu, v = np.zeros(n_sets, np.int64), np.zeros(n_sets), np.zeros(n_sets)
    for s in range(n_sets):
        seg = values[offsets[s]:offsets[s + 1]]
        c[s] = len(seg)
        mu[s] = seg.mean() if len(seg) else 0.0
        v[s] = seg.var(ddof=1) if len(seg) > 1 else 0.0
    return c, mu, v


@pytest.mark.parametrize("world", [1, 2, 3, 5, 7])
def test_combine_moments_matches_whole_batch(world):
    rng = np.random.default_rng(world)
    counts = [0, 1, 2, 7, 1000, 3, 0, 12345]
    off = W.offsets_from_counts(counts)
    y = rng.lognormal(0.1, 0.4, int(off[-1])) + 5.0       # an offset mean: the merge must not cancel
    parts = []
    for r in range(world):
        first, n = sharding.rank_range(int(off[-1]), world, r)
        local = np.clip(off - first, 0, n)
        parts.append(_set_moments(y[first:first + n], local))
    c, mu, v = sharding.combine_moments(*[np.array([p[i] for p in parts]) for i in range(3)])
    wc, wmu, wv = _set_moments(y, off)
    assert np.array_equal(c, wc)
    assert np.allclose(mu, wmu, rtol=1e-13, atol=0)
    assert np.allclose(v, wv, rtol=1e-10, atol=0)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _job():
    """A small batch: 4 GBM parameter sets with uneven path counts, a 4->50x4->7 network."""
    counts = [700, 1, 1300, 333]
    return dict(P=W.xavier_params(4, 7, seed=0), theta=W.gbm_online_thetas(4), Y0=np.array([1.0, 0.8, 1.2, 0.9]),
                off=W.offsets_from_counts(counts), T=2.0, n_steps=6, m=7, seed=5)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        j = _job()

        def compute(first, n):
            idx = np.arange(first, first + n)
            yt = oracle.seven_league_paths(oracle.MODEL_MLP, j["P"], j["theta"], j["Y0"], j["off"], j["T"],
                                           j["n_steps"], j["m"], j["seed"], idx=idx, d_in=4)
            compute.yt = yt
            c, mu, v = _set_moments(yt, np.clip(j["off"] - first, 0, n))
            return torch.as_tensor(c), torch.as_tensor(mu), torch.as_tensor(v)

        r = sharding.simulate_sharded(0, None, torch.as_tensor(j["theta"]), torch.as_tensor(j["Y0"]),
                                      torch.as_tensor(j["off"]), j["T"], j["n_steps"], j["m"], j["seed"],
                                      compute=compute)
        q.put((rank, r["first"], r["n_paths"], compute.yt, r["count"], r["mean"], r["var"]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_whole_batch(orc):
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    j = _job()
    whole = orc.seven_league_paths(orc.MODEL_MLP, j["P"], j["theta"], j["Y0"], j["off"], j["T"], j["n_steps"], j["m"],
                                   j["seed"], d_in=4)
    assert [g[1] for g in got] == [0, got[0][2]] and got[0][2] + got[1][2] == int(j["off"][-1])
    assert got[0][2] > int(j["off"][2]) > got[0][1]          # set 2 is split between the ranks
    assert np.array_equal(np.concatenate([g[3] for g in got]), whole)
    wc, wmu, wv = _set_moments(whole, j["off"])
    for g in got:                                            # every rank has the same combined moments
        assert np.array_equal(g[4], wc)
        assert np.allclose(g[5], wmu, rtol=1e-13, atol=1e-15)
        assert np.allclose(g[6], wv, rtol=1e-10, atol=1e-15)
    assert np.array_equal(got[0][5], got[1][5]) and np.array_equal(got[0][6], got[1][6])

"""One batched 7L call split across ranks (one process per GPU).

The method's paths are independent -- Algorithm I runs steps 3-6 per path and
collects the paths afterwards (steps 4 and 7) -- and every normal is a
counter-based Philox draw keyed by (set, path within the set, step).  So a
batch splits into contiguous ranges of its flat path list without changing a
single path: rank r runs its range through seven_league_simulate_range and
gets exactly the values the one-GPU call gives for those paths.  The only
exchange is the per-set partial moments (count, mean, variance in FP64),
gathered from every rank and combined in rank order, so every rank ends with
the same, deterministic per-set mean and variance.

Ranges are balanced by path count: every path costs the same n_steps network
evaluations, whatever its set.
"""
from __future__ import annotations

import numpy as np


def rank_range(total_paths: int, world: int, rank: int) -> tuple[int, int]:
    """(first_path, n_paths) of `rank`'s contiguous share of `total_paths` flat paths."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of world %d" % (rank, world))
    lo = total_paths * rank // world
    hi = total_paths * (rank + 1) // world
    return lo, hi - lo


def combine_moments(counts, means, variances):
    """Per-set count, mean and unbiased variance of the union of the ranks' paths.

    counts, means, variances: arrays [world, n_sets] in rank order (a rank's mean is 0
    without paths, its variance 0 with fewer than two).  The ranks are merged one after
    the other with the pairwise update of Chan, Golub and LeVeque (mean shift times the
    product of the counts), in FP64 and in rank order, so the result does not depend on
    how the partials were gathered."""
    counts = np.asarray(counts, dtype=np.float64)
    means = np.asarray(means, dtype=np.float64)
    variances = np.asarray(variances, dtype=np.float64)
    n = np.zeros(counts.shape[1])
    mean = np.zeros(counts.shape[1])
    m2 = np.zeros(counts.shape[1])
    for r in range(counts.shape[0]):
        nb = counts[r]
        m2b = np.where(nb > 1, variances[r] * np.maximum(nb - 1, 0), 0.0)
        nab = n + nb
        with np.errstate(invalid="ignore", divide="ignore"):
            delta = means[r] - mean
            frac = np.where(nab > 0, nb / np.where(nab > 0, nab, 1.0), 0.0)
            mean = np.where(nb > 0, mean + delta * frac, mean)
            m2 = np.where(nb > 0, m2 + m2b + delta * delta * n * frac, m2)
        n = nab
    var = np.where(n > 1, m2 / np.maximum(n - 1, 1), 0.0)
    return n.astype(np.int64), mean, var


def _world(group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(group), dist.get_rank(group)
    return 1, 0


def gather_partials(count, mean, var, group=None):
    """All ranks' (count, mean, var) tensors [n_sets] stacked in rank order: numpy
    arrays [world, n_sets].  One all-gather of a [3, n_sets] FP64 tensor, on the device the
    tensors live on (NCCL on GPUs, gloo on the host)."""
    import torch
    import torch.distributed as dist
    part = torch.stack([count.to(torch.float64), mean.to(torch.float64), var.to(torch.float64)])
    world, _ = _world(group)
    if world > 1 and part.is_cuda and dist.get_backend(group) != "nccl":
        part = part.cpu()              # gloo gathers host tensors
    if world == 1:
        parts = [part]
    else:
        parts = [torch.empty_like(part) for _ in range(world)]
        dist.all_gather(parts, part, group=group)
    a = torch.stack(parts).cpu().numpy()
    return a[:, 0], a[:, 1], a[:, 2]


def simulate_sharded(model, net, theta, Y0, path_offsets, T, n_steps, m, seed, total_paths=None,
                     group=None, compute=None, **range_kwargs):
    """This rank's share of one batched 7L call, and the whole batch's per-set moments.

    theta, Y0 and path_offsets describe the whole batch on every rank.  compute(first, n) runs
    the range and returns (count, mean, var) tensors [n_sets]; by default it is the library's
    seven_league_simulate_range on this rank's GPU (range_kwargs go to it: out_YT, out_grid, ws,
    stream).  Returns a dict with the range (first, n_paths), the combined per-set count, mean
    and var (numpy, identical on every rank) and the library's workspace (None for a custom
    compute)."""
    world, rank = _world(group)
    if total_paths is None:
        total_paths = int(path_offsets[-1].item())
    first, n = rank_range(int(total_paths), world, rank)
    ws = None
    if compute is None:
        import torch
        from . import seven_league_simulate_range
        n_sets = path_offsets.numel() - 1
        dev = theta.device
        count = torch.empty(n_sets, dtype=torch.int64, device=dev)
        mean = torch.empty(n_sets, dtype=torch.float64, device=dev)
        var = torch.empty(n_sets, dtype=torch.float64, device=dev)
        ws = seven_league_simulate_range(model, net, theta, Y0, path_offsets, T, n_steps, m, seed, first, n,
                                         out_mean=mean, out_var=var, out_count=count, **range_kwargs)
    else:
        count, mean, var = compute(first, n)
    c, mu, v = gather_partials(count, mean, var, group)
    tc, tm, tv = combine_moments(c, mu, v)
    return {"first": first, "n_paths": n, "count": tc, "mean": tm, "var": tv, "ws": ws}

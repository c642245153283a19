"""Sharding of independent paths over processes (one per GPU).

Paths are independent, so a tally shards by contiguous path-id ranges with
no exchange during tracing; the only collective is one reduction of the
per-rank FP64 sums at the end.  An image shards by pixels (every world-th
pixel of the claim order per rank, which keeps the ranks' loads even); a
flux by contiguous path-id ranges.  Online training of the proposal network
is data-parallel: one gradient average per Adam step (average_gradient).
The reduction gathers every rank's sums and adds them in rank order, so its
result is the same on every rank and from run to run, whatever the
transport (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations

import numpy as np

# Odd 64-bit constant (golden ratio) spacing replica seeds apart.
_SEED_STRIDE = 0x9E3779B97F4A7C15


def shard_range(total: int, rank: int, world: int, align: int = 1):
    """Contiguous [begin, end) of `total` path ids for `rank` of `world`,
    with interior boundaries on multiples of `align`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %d of %d" % (rank, world))
    if total < 0 or align < 1:
        raise ValueError("bad total or alignment")
    units = -(-total // align)
    lo = units * rank // world
    hi = units * (rank + 1) // world
    return min(lo * align, total), min(hi * align, total)


def image_shard_pixels(npix: int, rank: int, world: int):
    """Pixels of `rank`'s shard of an image traced in raster order
    (mcrt_trace_opts shard_index / shard_count with MCRT_ORDER_RASTER):
    every world-th pixel starting at rank.  With the cost order the library
    interleaves the same way over its claim order instead."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank %d of %d" % (rank, world))
    return np.arange(rank, npix, world, dtype=np.int64)


def combine_image(s1, s2, n_per_pixel, group=None):
    """One image from its shards: every rank holds per-pixel FP64 sums
    (Sum x, Sum x^2) of its own pixels (zeros elsewhere); the sums are added
    in rank order and the mean and standard error formed from them, the same
    on every rank."""
    t1, t2 = reduce_sums([s1, s2], group=group)
    m, se = mean_se(t1, t2, np.full(np.shape(t1), float(n_per_pixel)))
    return t1, t2, m, se


def replica_seed(seed: int, rank: int) -> int:
    """Seed of an independent replica on `rank` (distinct Philox keys)."""
    return (seed + rank * _SEED_STRIDE) % (1 << 64)


def reduce_sums(arrays, group=None):
    """Sum equally shaped FP64 arrays (e.g. Sum x, Sum x^2, N per tally
    entry) over all ranks in rank order; every rank gets the same result."""
    import torch
    import torch.distributed as dist
    flat = np.concatenate([np.ascontiguousarray(a, dtype=np.float64).ravel() for a in arrays])
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.from_numpy(flat).to(dev)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    total = parts[0].clone()
    for p in parts[1:]:
        total += p
    total = total.cpu().numpy()
    out, off = [], 0
    for a in arrays:
        n = np.asarray(a).size
        out.append(total[off:off + n].reshape(np.shape(a)))
        off += n
    return out


def average_gradient(grad, counts, group=None):
    """Data-parallel training of the proposal network: each rank holds the
    gradient of its own mean loss over `counts` records; the gradient of the
    mean loss over all ranks' records is the count-weighted average.  The
    ranks' gradients are gathered and combined in rank order in FP64, so
    every rank gets the same result (which it then applies with
    Proposal.apply_gradient, keeping the copies of the network equal)."""
    g = np.ascontiguousarray(grad, dtype=np.float64).ravel()
    weighted, n = reduce_sums([g * float(counts), np.array([float(counts)])], group=group)
    if not n[0] > 0:
        raise ValueError("no training records on any rank")
    return (weighted / n[0]).astype(np.float32)


def max_over_ranks(x: float, group=None) -> float:
    """Largest value of x over all ranks (step times)."""
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def mean_se(s1, s2, n):
    """Mean and standard error from Sum x, Sum x^2 and the count."""
    s1 = np.asarray(s1, dtype=np.float64)
    s2 = np.asarray(s2, dtype=np.float64)
    n = np.asarray(n, dtype=np.float64)
    m = s1 / n
    var = np.maximum(s2 / n - m * m, 0.0)
    return m, np.where(n > 1, np.sqrt(var / np.maximum(n - 1, 1)), 0.0)

"""Sharding paths over ranks and combining their moments (torch.distributed).

Stochastic paths and independent instances need no exchange while they are
integrated (XMDS2 runs its paths as separate MPI processes, Sec. 2.5): each
rank advances a contiguous range of global path indices, and the Philox
counters carry the global index (``path_offset``), so a path's noise, and
therefore its result, does not depend on how the ensemble is split.  The only
collective is the combination of the ensemble moments, once per sample set,
in FP64.  Works with any process group (NCCL for device tensors, gloo for
host tensors); no arithmetic of the time step happens here.
"""
from __future__ import annotations


def shard(total: int, rank: int, world: int) -> tuple[int, int]:
    """(path_offset, count) of rank's contiguous share of `total` paths: the
    first total % world ranks take one path more."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("need 0 <= rank < world and total >= 0")
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def combine_per_point(per_point, count: int, total: int, group=None):
    """Ensemble means over all ranks' paths from each rank's means over its own
    `count` paths (the per-point buffer of xsde_moments, [nsamp][npts][2]):
    sum_r (count_r / total) mean_r, summed in place by an all-reduce."""
    import torch.distributed as dist
    per_point.mul_(count / total)
    dist.all_reduce(per_point, op=dist.ReduceOp.SUM, group=group)
    return per_point


def gather_per_path(per_path, counts, group=None):
    """All ranks' per-path values ([nsamp][count_r][2] each) in global path
    order, [nsamp][total][2]; counts[r] is rank r's path count."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    if len(counts) != world:
        raise ValueError("one count per rank")
    width = max(counts)
    padded = per_path.new_zeros((per_path.shape[0], width, per_path.shape[2]))
    padded[:, :per_path.shape[1]] = per_path
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([p[:, :c] for p, c in zip(parts, counts)], dim=1)

"""Row sharding of a query batch over ranks (one process per GPU).

Rows are independent (each row's outputs depend only on that row and the
scene), so a batch splits into contiguous row ranges, one per rank, each
answered against that rank's own resident copy of the scene; no collective
runs on the data path.  Ranges keep groups of `group_size` rows whole, so
per-group outputs are computed where their rows are.  `gather_rows` brings the
per-rank results together on every rank (the host-side assembly step).
"""
from __future__ import annotations


def shard_range(Q: int, group_size: int, rank: int, world: int) -> tuple[int, int]:
    """Row range [start, stop) of `rank`: whole groups, split as evenly as
    possible (the first ranks take one group more when they do not divide)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if Q < 0:
        raise ValueError("Q must be >= 0")
    G = max(1, int(group_size))
    ngroups = (Q + G - 1) // G
    base, extra = divmod(ngroups, world)
    g0 = rank * base + min(rank, extra)
    g1 = g0 + base + (1 if rank < extra else 0)
    return min(Q, g0 * G), min(Q, g1 * G)


def gather_rows(local, Q: int, group_size: int, world: int, group=None):
    """Concatenate every rank's rows (a 1-D or 2-D torch tensor holding the
    rows of shard_range for that rank) into the full [Q, ...] result on every
    rank, over torch.distributed (any backend; CPU tensors for gloo)."""
    import torch
    import torch.distributed as dist
    sizes = [shard_range(Q, group_size, r, world) for r in range(world)]
    n_max = max(b - a for a, b in sizes)
    pad = torch.zeros((n_max,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([bufs[r][: b - a] for r, (a, b) in enumerate(sizes)])

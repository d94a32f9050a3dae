"""Data-parallel replicas: poses are independent, so N GPUs run N model replicas.

The paper splits a job's poses across ranks by rank index and collects
identifiers and predictions once at the end (Section 4.2).  Here each rank
scores a contiguous shard of the pose list on its own GPU; the only
collective is the end-of-job gather of the affinities, outside the scoring
path.  These helpers are host logic only (no GPU work).
"""

from __future__ import annotations

import numpy as np


def shard_range(n_items: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) of n_items for `rank` of `world`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_items, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_affinities(local: np.ndarray, n_items: int, group=None) -> np.ndarray:
    """All-gather every rank's shard of affinities into the global order (end of a job).

    Uses torch.distributed with whatever backend the process group has (gloo on
    CPU, nccl on GPUs); shards are padded to a common length for the collective.
    """
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    b, e = shard_range(n_items, rank, world)
    assert len(local) == e - b, "local shard has the wrong length"
    width = -(-n_items // world)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = torch.full((width,), float("nan"), dtype=torch.float32, device=dev)
    buf[: len(local)] = torch.as_tensor(np.asarray(local, dtype=np.float32), device=dev)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    out = np.empty(n_items, dtype=np.float32)
    for r in range(world):
        rb, re_ = shard_range(n_items, r, world)
        out[rb:re_] = parts[r][: re_ - rb].cpu().numpy()
    return out

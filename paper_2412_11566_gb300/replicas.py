"""Replica parallelism for the LS solves (one process per GPU).

The solves of different microstructures (and load cases) share nothing, so
the path has no exchange step and needs no collective on the data path: each
rank takes a contiguous slice of the items, solves them on its own GPU, and
rank 0 gathers the 36 C_eff doubles per item. Only the bookkeeping below
crosses ranks (a gather of results and the maximum of the timed region)."""
from __future__ import annotations

import numpy as np


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous slice of items of this rank; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def gather_ceff(local: np.ndarray, n_items: int, rank: int, world: int):
    """Assemble the (n_items, 6, 6) C_eff array on rank 0 from each rank's
    (len(shard), 6, 6) slice; other ranks get None. Uses torch.distributed
    (any backend) when world > 1."""
    local = np.asarray(local, dtype=np.float64).reshape(-1, 6, 6)
    if world == 1:
        return local.copy()
    import torch
    import torch.distributed as dist
    sizes = [len(shard(n_items, r, world)) for r in range(world)]
    if local.shape[0] != sizes[rank]:
        raise ValueError("local slice does not match this rank's shard")
    width = max(sizes)
    buf = torch.zeros((width, 36), dtype=torch.float64)
    buf[: sizes[rank]] = torch.from_numpy(local.reshape(-1, 36))
    outs = [torch.zeros_like(buf) for _ in range(world)] if rank == 0 else None
    dist.gather(buf, gather_list=outs, dst=0)
    if rank != 0:
        return None
    return np.concatenate([o[: s].numpy() for o, s in zip(outs, sizes)]).reshape(n_items, 6, 6)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank scalar (the timed region's duration)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device=None) -> float:
    """Sum of a per-rank scalar (solves counted by every rank)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

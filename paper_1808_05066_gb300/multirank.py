"""Host-side helpers for runs with one process per GPU (torchrun).

Elements are independent in assemble + condense, so ranks need no data exchange: each
rank owns a contiguous slab of elements (or, in the weak-scaling bench, a replica of the
workload) and the ranks only agree on timing (max over ranks). Works with the gloo
(CPU) and NCCL (GPU) backends."""
from __future__ import annotations

import os


def world():
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 otherwise)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def partition(n_units: int, rank: int, world_size: int):
    """Contiguous slab [start, start + count) of n_units for this rank; slabs differ in
    size by at most one and cover every unit exactly once."""
    base, extra = divmod(n_units, world_size)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a scalar over all ranks of the default process group (identity when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

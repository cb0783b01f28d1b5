"""Several GPUs of one node: one process per GPU (launched by torchrun), each
running the path on its own units -- groups, jobs, requests -- with no
collective on the data path, since the units are independent.  The only
collectives are the timing ones: a barrier before the timed region and the
maximum of the per-rank times after it.  The same code runs over NCCL on GPUs
and over gloo on CPU processes (the tests)."""
from __future__ import annotations

import os


def world_info():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str):
    """Join the process group of the launcher's environment (no-op for one process)."""
    import torch.distributed as dist
    _, world, _ = world_info()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)


def finish():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()


def barrier():
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks (the whole job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def rank_seed(seed: int, rank: int) -> int:
    """Data seed of a rank: every rank draws its own units of the same shape
    (rank 0 keeps the base seed, so its units are the one-GPU workload)."""
    return seed + 1_000_003 * rank


def shard(n_units: int, world: int, rank: int):
    """Contiguous block [start, stop) of n_units for this rank; the blocks of
    all ranks partition range(n_units) and differ in size by at most one."""
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)

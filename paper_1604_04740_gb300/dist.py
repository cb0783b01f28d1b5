"""Several GPUs of one node: one process per GPU (launched by torchrun).

Two ways to spread the path over ranks:
  - by units (the benchmark's way): each rank runs the whole path on its own
    groups, jobs or requests with no collective on the data path, since the
    units are independent; the only collectives are the timing ones (a
    barrier before the timed region, the maximum of the per-rank times after);
  - by streams (the paper's own distribution, one stream per processing core,
    Sec. I and Sec. III): rank m computes only delta_m = eps_m op g; the
    extraction then needs every stream's word of a position in one place, so
    the ranks exchange their results by position block (one all-to-all) and
    each extracts and checks its block.  A rank that fails (fail-stop) is
    found by a host-side heartbeat, and the survivors exchange among
    themselves and rebuild every output without it (Prop. 3).
The same code runs over NCCL on GPUs and over gloo on CPU processes (the
tests); the extraction itself is the library's (ne_extract / ne_recover on
the gathered block)."""
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


# ---- one stream per rank: the exchange by position block ---------------------------------

def stream_groups(world: int):
    """The process groups the survivors use after one rank has failed: entry d
    holds every rank but d.  Collective: every rank calls it once, while all
    are alive (after init, before the first exchange)."""
    import torch.distributed as dist
    return {d: dist.new_group([r for r in range(world) if r != d]) for d in range(world)}


def heartbeat(store, step: int, rank: int, world: int, timeout_s: float = 2.0):
    """Fail-stop detection on the host before an exchange: every live rank
    posts the key hb/<step>/<rank> in the shared store, then waits up to
    timeout_s for each other rank's key.  Returns the ranks whose key never
    appeared (the failed ones), the same list on every live rank when the
    failed ranks stopped before posting."""
    import datetime
    store.set(f"hb/{step}/{rank}", "1")
    dead = []
    for r in range(world):
        if r == rank:
            continue
        try:
            store.wait([f"hb/{step}/{r}"], datetime.timedelta(seconds=timeout_s))
        except Exception:
            dead.append(r)
    return dead


def exchange_streams(delta_m, rank: int, world: int, dead=None, groups=None):
    """All-to-all of the streams' results by position block.

    delta_m: this rank's stream m = rank, all n positions (1-D tensor, on the
    rank's device).  The positions are cut into P blocks of ceil(n / P), P the
    number of live ranks (world, or world - 1 with dead = d); live rank number
    p (in rank order) receives block p of every live stream.  Returns (block,
    start, stop): block is [world, stop - start] with row m holding
    delta_m[start:stop] (row d zero: the failed stream, never to be read --
    recover with r_lost = d)."""
    import torch
    import torch.distributed as dist
    live = [r for r in range(world) if r != dead] if dead is not None else list(range(world))
    P = len(live)
    p = live.index(rank)
    n = delta_m.numel()
    B = -(-n // P) if n else 0
    send = torch.zeros(P * B, dtype=delta_m.dtype, device=delta_m.device)
    send[:n] = delta_m.reshape(-1)
    recv = torch.empty_like(send)
    if P > 1:
        dist.all_to_all_single(recv, send, group=None if dead is None else groups[dead])
    else:
        recv.copy_(send)
    start, stop = min(p * B, n), min((p + 1) * B, n)
    block = torch.zeros((world, stop - start), dtype=delta_m.dtype, device=delta_m.device)
    recv = recv.view(P, B)
    for q, r in enumerate(live):
        block[r] = recv[q, :stop - start]
    return block, start, stop

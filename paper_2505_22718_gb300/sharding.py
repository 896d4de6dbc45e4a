"""Walker sharding across ranks (one process per GPU).

Parameter points are independent, so ranks split them with no exchange on the data path: each
rank evaluates a contiguous block of walkers.  The only collectives are outside the hot path: the
slowest rank's time for benchmarking and, for samplers that want every chain's spectra on every
rank, an all-gather of the results.  Works with any torch.distributed backend (NCCL on GPUs, gloo
on CPU).
"""
from __future__ import annotations


def shard(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """(first walker, number of walkers) of `rank`: contiguous blocks whose sizes differ by at most
    one, the larger blocks first."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar (e.g. elapsed milliseconds) over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_blocks(block, n_total: int):
    """All-gather of per-rank result blocks (first dimension = the rank's walkers, in rank order)
    into one tensor of n_total rows on every rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return block
    world = dist.get_world_size()
    sizes = [shard(n_total, world, r)[1] for r in range(world)]
    width = max(sizes)
    pad = torch.zeros((width,) + tuple(block.shape[1:]), dtype=block.dtype, device=block.device)
    pad[:block.shape[0]] = block
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)], dim=0)

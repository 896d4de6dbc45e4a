"""Sharding across ranks (one process per GPU).

Walkers: parameter points are independent, so ranks split them with no exchange on the data path:
each rank evaluates a contiguous block of walkers.  The only collectives are outside the hot path:
the slowest rank's time for benchmarking and, for samplers that want every chain's spectra on every
rank, an all-gather of the results.

Multipoles: one evaluation too large for one GPU splits by multipole.  Every rank runs the FFTLog
(Eq. 3.2) for all tracers, which is cheap, and the contraction, quadrature and reverse mode for its
own contiguous block of multipoles, whose C_ell are disjoint (Eq. 2.1 is a separate k-integral per
multipole).  The gradients P_bar, A_bar and W_bar are sums over multipoles, so one sum all-reduce
of the three forms the full gradient.

Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
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


def ell_block(n_ell: int, world: int, rank: int) -> tuple[int, int]:
    """(first multipole index, count) of `rank` when one evaluation splits its n_ell multipoles
    across `world` ranks: contiguous blocks whose sizes differ by at most one.  Every rank needs at
    least one multipole."""
    if world > n_ell:
        raise ValueError("more ranks than multipoles")
    return shard(n_ell, world, rank)


def reduce_gradients(*grads):
    """Sum over ranks of the reverse mode's outputs (P_bar, A_bar, W_bar, each a sum over the
    rank's multipoles), packed into one buffer for a single all-reduce.  Returns the summed
    tensors (the inputs themselves when no process group is running)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return grads
    flat = torch.cat([g.reshape(-1) for g in grads])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    out, off = [], 0
    for g in grads:
        n = g.numel()
        out.append(flat[off:off + n].view_as(g))
        off += n
    return tuple(out)

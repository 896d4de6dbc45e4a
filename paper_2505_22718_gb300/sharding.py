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
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return block
    world = dist.get_world_size()
    return gather_blocks_sized(block, [shard(n_total, world, r)[1] for r in range(world)])


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


def library_block(setup, C_bar, precision, device=0):
    """One rank's share of a multipole-split evaluation through the library: a context on
    `device` for the rank's block of the multipole list (setup["ells"]), forward and reverse mode.
    Returns numpy arrays (C [n_l][N_tr][N_tr], P_bar [N_k], amp_bar [N_tr], W_bar [N_tr][N])."""
    from .api import Context
    ctx = Context(device, 0)
    try:
        ctx.set_grids(setup["chi_min"], setup["chi_max"], setup["N"], setup["k"], setup["ells"],
                      setup["knots"])
        ctx.set_tracers(setup["kind"], setup["fft_bias"], setup.get("taper_chi"),
                        setup.get("taper_c"))
        ctx.set_windows(setup["W"], setup["D"], setup.get("B"))
        ctx.set_power(setup["P"], setup["amp"])
        C = ctx.compute_cl(precision)
        Pb, Ab, Wb = ctx.vjp(C_bar, precision)
    finally:
        ctx.close()
    return C, Pb[0], Ab[0], Wb[0]


def evaluate_ell_split(setup, C_bar, precision=0, block=None, device=0):
    """One evaluation (one parameter point) split by multipole across the process group.

    setup: dict with chi_min, chi_max, N, k, ells (the whole multipole list), knots, kind,
    fft_bias, W [N_tr][N], D [N_I][N], P [N_k], amp [N_tr] and optionally B, taper_chi, taper_c.
    C_bar: the cotangent of the whole evaluation, [N_ell][N_tr][N_tr].
    Each rank evaluates its contiguous block of multipoles (ell_block) with `block`
    (default library_block: the C ABI on `device`), then the C_ell blocks are all-gathered along
    the multipoles (gather_blocks) and the gradients, which are sums over multipoles, are summed
    with one all-reduce (reduce_gradients).  Every rank returns the full
    (C, P_bar, amp_bar, W_bar) as CPU float64 tensors.  Without a process group it evaluates
    everything on this process."""
    import numpy as np
    import torch
    import torch.distributed as dist
    world, rank = 1, 0
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(), dist.get_rank()
    ells = np.asarray(setup["ells"])
    first, count = ell_block(len(ells), world, rank)
    mine = dict(setup)
    mine["ells"] = np.ascontiguousarray(ells[first:first + count])
    run = block or (lambda su, cb, p: library_block(su, cb, p, device))
    C, Pb, Ab, Wb = run(mine, np.ascontiguousarray(np.asarray(C_bar)[first:first + count]), precision)
    # NCCL exchanges device tensors, gloo host tensors
    on = torch.device("cuda", device) if world > 1 and dist.get_backend() == "nccl" else torch.device("cpu")
    as_t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=on)  # noqa: E731
    C_all = gather_blocks_sized(as_t(C), [ell_block(len(ells), world, r)[1] for r in range(world)])
    Pb, Ab, Wb = reduce_gradients(as_t(Pb), as_t(Ab), as_t(Wb))
    return C_all.cpu(), Pb.cpu(), Ab.cpu(), Wb.cpu()


def gather_blocks_sized(block, sizes):
    """All-gather of per-rank blocks of the given first-dimension sizes (rank order), concatenated
    on every rank (the block itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return block
    width = max(sizes)
    pad = torch.zeros((width,) + tuple(block.shape[1:]), dtype=block.dtype, device=block.device)
    pad[:block.shape[0]] = block
    parts = [torch.empty_like(pad) for _ in range(len(sizes))]
    dist.all_gather(parts, pad)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)], dim=0)

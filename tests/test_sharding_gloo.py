"""The multi-rank path on CPU: walker shards across two gloo ranks, the max-over-ranks timing
reduction and the all-gather of per-rank results (no GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_2505_22718_gb300.sharding import shard


def test_shard_partitions_walkers():
    for n in (0, 1, 7, 256, 257):
        for world in (1, 2, 3, 8):
            blocks = [shard(n, world, r) for r in range(world)]
            starts = [b[0] for b in blocks]
            counts = [b[1] for b in blocks]
            assert sum(counts) == n
            assert starts[0] == 0
            assert all(starts[r] + counts[r] == starts[r + 1] for r in range(world - 1))
            assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_total, out):
    import torch
    import torch.distributed as dist
    from paper_2505_22718_gb300.sharding import gather_blocks, max_over_ranks, shard
    from workloads import make_workload
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    first, count = shard(n_total, world, rank)
    # a rank builds only its own walkers; a per-walker summary stands in for its C_ell
    w = make_workload("walkers", n_walkers=count, first_walker=first)
    block = torch.tensor(np.stack([w.P[i][:4] * w.amp[i][0] for i in range(count)]))
    full = gather_blocks(block, n_total)
    t = max_over_ranks(10.0 + rank)
    dist.barrier()
    if rank == 0:
        out.put((full.numpy(), t))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process():
    import torch.multiprocessing as mp
    from workloads import make_workload
    n_total, world = 5, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_total, q)) for r in range(world)]
    for p in procs:
        p.start()
    full, t = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = make_workload("walkers", n_walkers=n_total)
    ref = np.stack([w.P[i][:4] * w.amp[i][0] for i in range(n_total)])
    assert np.array_equal(full, ref)
    assert t == 11.0

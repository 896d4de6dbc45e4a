"""The multi-rank path on CPU: walker shards across two gloo ranks, the max-over-ranks timing
reduction and the all-gather of per-rank results; one evaluation split by multipole across two
gloo ranks, with the oracle standing in for each rank's compute (no GPU)."""
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


def _ell_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from oracle import fftlog as O
    from paper_2505_22718_gb300.sharding import ell_block, gather_blocks, reduce_gradients
    from workloads import make_workload
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    w = make_workload("tiny2")
    first, count = ell_block(len(w.ells), world, rank)
    ells = w.ells[first:first + count]
    Cb = np.random.default_rng(5).standard_normal((len(w.ells), w.n_tr, w.n_tr))[first:first + count]
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, ells, w.knots, w.kind, w.fft_bias)
    f = O.forward(g, w.W, w.D, w.P, w.amp, w.B)
    Pb, Ab, Wb, _ = O.vjp(g, f, Cb, w.W, w.D, w.P, w.amp, w.B)
    C = gather_blocks(torch.tensor(f["C"]), len(w.ells))
    Pb, Ab, Wb = reduce_gradients(torch.tensor(Pb), torch.tensor(Ab), torch.tensor(Wb))
    dist.barrier()
    if rank == 0:
        out.put((C.numpy(), Pb.numpy(), Ab.numpy(), Wb.numpy()))
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_evaluation_by_ell():
    """C_ell blocks gathered along the multipoles and the per-rank gradients summed equal one
    process's full evaluation."""
    import torch.multiprocessing as mp
    from oracle import fftlog as O
    from paper_2505_22718_gb300.sharding import ell_block
    from workloads import make_workload
    w = make_workload("tiny2")
    assert [ell_block(20, 3, r) for r in range(3)] == [(0, 7), (7, 7), (14, 6)]
    with pytest.raises(ValueError):
        ell_block(2, 3, 0)
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ell_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    C, Pb, Ab, Wb = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    Cb = np.random.default_rng(5).standard_normal((len(w.ells), w.n_tr, w.n_tr))
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind, w.fft_bias)
    f = O.forward(g, w.W, w.D, w.P, w.amp, w.B)
    Pbo, Abo, Wbo, _ = O.vjp(g, f, Cb, w.W, w.D, w.P, w.amp, w.B)
    assert np.max(np.abs(C - f["C"])) <= 1e-13 * np.abs(f["C"]).max()
    for a, b in ((Pb, Pbo), (Ab, Abo), (Wb, Wbo)):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.abs(b).max()

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


def _oracle_cl(w, i):
    """The oracle's C_ell of walker i of a walkers workload (numpy.fft form of Eq. 3.2)."""
    from oracle import fftlog as O
    g = O.Grids(w.N, w.chi_min, w.chi_max, w.k, w.ells, w.knots, w.kind, w.fft_bias, fft="numpy")
    return O.forward(g, w.W[i], w.D, w.P[i], w.amp[i], w.B)["C"]


def _worker(rank, world, port, n_total, out):
    import torch
    import torch.distributed as dist
    from paper_2505_22718_gb300.sharding import gather_blocks, max_over_ranks, shard
    from workloads import make_workload
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    first, count = shard(n_total, world, rank)
    # a rank builds only its own walkers and evaluates their C_ell (the oracle stands in for the
    # GPU compute of each rank)
    w = make_workload("walkers", n_walkers=count, first_walker=first)
    block = torch.tensor(np.stack([_oracle_cl(w, i) for i in range(count)]))
    full = gather_blocks(block, n_total)
    t = max_over_ranks(10.0 + rank)
    dist.barrier()
    if rank == 0:
        out.put((full.numpy(), t))
    dist.destroy_process_group()


def test_two_gloo_ranks_match_one_process():
    import torch.multiprocessing as mp
    from workloads import make_workload
    n_total, world = 3, 2
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
    ref = np.stack([_oracle_cl(w, i) for i in range(n_total)])
    assert np.array_equal(full, ref)
    assert t == 11.0


def _oracle_block(su, Cb, precision):
    """A rank's compute in the multipole split, with the oracle standing in for the library."""
    from oracle import fftlog as O
    g = O.Grids(su["N"], su["chi_min"], su["chi_max"], su["k"], su["ells"], su["knots"], su["kind"],
                su["fft_bias"])
    f = O.forward(g, su["W"], su["D"], su["P"], su["amp"], su.get("B"))
    Pb, Ab, Wb, _ = O.vjp(g, f, Cb, su["W"], su["D"], su["P"], su["amp"], su.get("B"))
    return f["C"], Pb, Ab, Wb


def _setup(w):
    return dict(chi_min=w.chi_min, chi_max=w.chi_max, N=w.N, k=w.k, ells=w.ells, knots=w.knots,
                kind=w.kind, fft_bias=w.fft_bias, W=w.W, D=w.D, B=w.B, P=w.P, amp=w.amp)


def _ell_worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2505_22718_gb300.sharding import evaluate_ell_split
    from workloads import make_workload
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    w = make_workload("tiny2")
    Cb = np.random.default_rng(5).standard_normal((len(w.ells), w.n_tr, w.n_tr))
    # the end-to-end entry point: ell_block, the rank's block, gather_blocks, reduce_gradients
    C, Pb, Ab, Wb = evaluate_ell_split(_setup(w), Cb, block=_oracle_block)
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

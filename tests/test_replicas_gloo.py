"""Replica sharding of the sources, world_size 2 over gloo on CPU.

Each rank runs the oracle's truncated-solver sums on its own share of the
bulk and correction source ids; one sum over ranks of the three accumulators
must give the single-process TSM estimate (the rule the multi-GPU path uses,
with no collective on the data path before that final sum).  The max-over-
ranks timing reduction is checked alongside.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1401_6750_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    from oracle import lattice, momenta, tsm
    from paper_1401_6750_gb300 import replicas as rep
    from paper_1401_6750_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dims = (2, 2, 2, 4)
    kappa, mu, seed, n_lp, n_hp = 0.12, 0.05, 7, 5, 3
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 3), -1)
    moms = momenta.momentum_list(1)
    shape = (160, len(moms), dims[3])
    sums = [np.zeros(shape, complex) for _ in range(3)]
    f, c = rep.shard(n_lp, rank, world)
    for r in range(f, f + c):
        sums[0] += tsm.source_loops(u, dims, kappa, mu, seed, r, 1e-3, moms)[0]
    f, c = rep.shard(n_hp, rank, world)
    for r in range(n_lp + f, n_lp + f + c):
        sums[1] += tsm.source_loops(u, dims, kappa, mu, seed, r, 1e-10, moms)[0]
        sums[2] += tsm.source_loops(u, dims, kappa, mu, seed, r, 1e-3, moms)[0]
    total = [rep.sum_over_ranks(x) for x in sums]
    est = tsm.combine(total[0], n_lp, total[1], total[2], n_hp)
    tmax = rep.max_over_ranks(1.0 + rank)
    if rank == 0:
        np.save(os.path.join(out_dir, "est.npy"), est)
        np.save(os.path.join(out_dir, "tmax.npy"), np.array([tmax]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_covers_every_source_once():
    for n in (0, 1, 5, 32, 33):
        for world in (1, 2, 3, 8):
            ids = []
            for rank in range(world):
                f, c = replicas.shard(n, rank, world)
                ids.extend(range(f, f + c))
            assert ids == list(range(n))


def test_two_rank_split_and_sum_equals_single_process(tmp_path):
    from oracle import lattice, momenta, tsm
    from paper_1401_6750_gb300 import synth
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    est = np.load(tmp_path / "est.npy")
    dims = (2, 2, 2, 4)
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 3), -1)
    want, _ = tsm.tsm_loops(u, dims, 0.12, 0.05, 7, 5, 3, 1e-3, 1e-10, momenta.momentum_list(1))
    assert np.allclose(est, want, rtol=1e-12, atol=1e-14)
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.0

"""Two-rank (gloo, CPU) test of the pair sharding used by the batch path on N GPUs.

Each rank takes its longest-processing-time share of the pairs, computes it
(here with the CPU oracle: no GPU on this path), and the shards are gathered;
the union must be exactly the single-process result, every pair computed
once, and the per-rank loads balanced.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, ret):
    import torch.distributed as dist
    import oracle
    from paper_2404_05708_gb300 import shard, workloads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = workloads.ragged_int_batch(n_pairs=300, len_lo=4, len_hi=120, seed=33)
        idx = shard.shard_pairs(b.lengths(), b.pairs, rank, world)
        vals, _ = oracle.batch(b.points, b.offsets, b.pairs[idx], nthreads=1)
        full = shard.gather(vals, idx, b.pairs.shape[0])
        cells = float(np.sum(b.lengths()[b.pairs[idx, 0]] * b.lengths()[b.pairs[idx, 1]]))
        total = shard.sum_over_ranks(cells)
        most = shard.max_over_ranks(cells)
        counts = [None] * world
        dist.all_gather_object(counts, int(idx.shape[0]))
        if rank == 0:
            ref, _ = oracle.batch(b.points, b.offsets, b.pairs, nthreads=1)
            ret.put((np.array_equal(full, ref), sum(counts), b.pairs.shape[0], total, most))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_rank_sharding_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    ret = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ret)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    same, n_done, n_total, total_cells, max_cells = ret.get(timeout=10)
    assert same
    assert n_done == n_total
    assert max_cells <= 0.51 * total_cells   # LPT keeps the two loads within 2 %


def test_lpt_assignment_properties():
    from paper_2404_05708_gb300 import shard
    rng = np.random.default_rng(3)
    costs = rng.integers(1, 1000, size=1000).astype(np.float64)
    for world in (1, 2, 3, 8):
        owner = shard.lpt_assign(costs, world)
        loads = np.bincount(owner, weights=costs, minlength=world)
        assert loads.sum() == costs.sum()
        assert loads.max() - loads.min() <= costs.max()

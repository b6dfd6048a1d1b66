"""The collective-free multi-process split, on CPU with gloo (world size 2)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2308_08417_gb300.sharding import max_over_ranks, shard_range


def test_shard_ranges_cover_the_batch_once():
    for B in (0, 1, 7, 64, 65536, 100001):
        for world in (1, 2, 3, 4, 8):
            spans = [shard_range(B, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == B
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2308_08417_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = W.plain_at_scale(96)
    b0, b1 = shard_range(wl.num_batch, rank, world)
    A = wl.matrix("csr").subset(np.arange(b0, b1))
    x, it, rel, st = oracle.solve_batch(A, wl.b[b0:b1], threads=1)
    # gather the shards to rank 0 (result collection, not part of the solve)
    parts = [None] * world
    dist.all_gather_object(parts, (b0, x, it))
    slow = max_over_ranks(float(rank + 1), dist)
    if rank == 0:
        out.put((parts, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_split_equals_single_solve():
    import oracle
    from paper_2308_08417_gb300 import workloads as W

    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    parts, slow = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = W.plain_at_scale(96)
    x, it, rel, st = oracle.solve_batch(wl.matrix("csr"), wl.b, threads=1)
    xs = np.concatenate([p[1] for p in sorted(parts, key=lambda t: t[0])])
    its = np.concatenate([p[2] for p in sorted(parts, key=lambda t: t[0])])
    assert np.array_equal(xs, x) and np.array_equal(its, it)
    assert slow == 2.0


def test_cost_shard_ranges_balance_uneven_batches():
    from paper_2308_08417_gb300.sharding import cost_shard_range

    rng = np.random.default_rng(5)
    for B in (0, 1, 9, 1000):
        costs = rng.lognormal(3.0, 1.5, B)
        for world in (1, 2, 3, 8):
            spans = [cost_shard_range(costs, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == B
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            if B >= 1000:  # every rank within one system's cost of its share
                share = costs.sum() / world
                for b0, b1 in spans:
                    assert abs(costs[b0:b1].sum() - share) <= costs.max()
    # equal costs: the plain split up to rounding
    for B, world in ((64, 2), (1000, 8), (7, 3)):
        for r in range(world):
            a, b = cost_shard_range(np.ones(B), r, world)
            c, d = shard_range(B, r, world)
            assert abs(a - c) <= 1 and abs(b - d) <= 1
    with pytest.raises(ValueError):
        cost_shard_range([1.0, -1.0], 0, 2)


def test_varbatch_slices_reassemble_the_batch():
    from paper_2308_08417_gb300 import workloads as W
    from paper_2308_08417_gb300.sharding import cost_shard_range

    vb = W.uneven(500)
    cost = (2 * vb.sys_nnz() + 14 * vb.sys_n()) * np.sqrt(vb.sys_n())
    parts = [vb.slice(*cost_shard_range(cost, r, 3)) for r in range(3)]
    assert sum(p.num_batch for p in parts) == vb.num_batch
    assert np.array_equal(np.concatenate([p.values for p in parts]), vb.values)
    assert np.array_equal(np.concatenate([p.b for p in parts]), vb.b)
    i = 0
    for p in parts:
        for j in range(p.num_batch):
            a, b = p.system(j), vb.system(i)
            assert a[0] is b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
            i += 1

"""Multi-rank host logic on CPU (gloo, world_size 2): sharding of independent
problems across ranks and the max-over-ranks timing reduction bench.py uses."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import gen
    from paper_2406_10849_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    probs = gen.batched_problems(seed=4000, num_trees=24, n_range=(16, 64))
    mine, idx = shard.shard_problems(probs, rank, world)
    load = sum(p.elements_per_half_step() for p in mine)
    t_max = shard.max_over_ranks(1.0 + rank, dist)
    total = shard.sum_over_ranks(load, dist)
    out[rank] = (idx, load, t_max, total)
    dist.barrier()
    dist.destroy_process_group()


def test_sharding_world2_gloo():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    idx0, load0, tmax0, tot0 = out[0]
    idx1, load1, tmax1, tot1 = out[1]
    assert sorted(idx0 + idx1) == list(range(24))
    assert not set(idx0) & set(idx1)
    assert tmax0 == tmax1 == 2.0
    assert tot0 == tot1 == load0 + load1
    assert max(load0, load1) / min(load0, load1) < 1.3


def _bench_share_worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_2406_10849_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    probs, idx = bench.batched_share(512, rank, world)
    edges = sum(p.num_edges for p in probs)
    elems = sum(p.elements_per_half_step() for p in probs)
    out[rank] = (idx, edges, elems, shard.sum_over_ranks(edges, dist), shard.max_over_ranks(elems, dist))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_batched_split_world2_gloo():
    """The batched benchmark's split at world size 2, as each rank builds it: the two
    ranks' trees are disjoint and cover the 512, the summed edge count (the numerator
    of the whole-job applies/s) equals the batch's, and the heavier rank carries
    within 1 % of half the plan elements (the time of a step is the max over ranks)."""
    import gen
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_bench_share_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    allp = gen.batched_problems(seed=4000, num_trees=512)
    (i0, e0, m0, tot0, mx0), (i1, e1, m1, tot1, mx1) = out[0], out[1]
    assert sorted(i0 + i1) == list(range(512)) and not set(i0) & set(i1)
    assert tot0 == tot1 == e0 + e1 == sum(p.num_edges for p in allp)
    total = sum(p.elements_per_half_step() for p in allp)
    assert m0 + m1 == total and mx0 == mx1 == max(m0, m1)
    assert max(m0, m1) <= 0.505 * total


def test_shard_range_covers_all():
    from paper_2406_10849_gb300 import shard
    for n in (0, 1, 7, 512):
        for w in (1, 2, 3, 8):
            spans = [shard.shard_range(n, r, w) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1

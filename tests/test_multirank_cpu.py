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
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    idx0, load0, tmax0, tot0 = out[0]
    idx1, load1, tmax1, tot1 = out[1]
    assert sorted(idx0 + idx1) == list(range(24))
    assert not set(idx0) & set(idx1)
    assert tmax0 == tmax1 == 2.0
    assert tot0 == tot1 == load0 + load1
    assert max(load0, load1) / min(load0, load1) < 1.3


def test_shard_range_covers_all():
    from paper_2406_10849_gb300 import shard
    for n in (0, 1, 7, 512):
        for w in (1, 2, 3, 8):
            spans = [shard.shard_range(n, r, w) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1

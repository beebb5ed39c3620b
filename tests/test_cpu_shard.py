"""Host logic of the multi-GPU path: bases are split across ranks with no
data-path collective; checked with world_size-2 gloo process groups."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1409_2556_gb300.shard import partition


def test_partition_covers_disjointly():
    for n in (0, 1, 5, 27, 64):
        for w in (1, 2, 3, 8):
            parts = [partition(n, r, w) for r in range(w)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        partition(3, 2, 2)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = partition(27, rank, world)
    t = torch.zeros(27)
    t[mine] = 1.0
    dist.all_reduce(t)                      # test-only check that every basis is owned once
    tm = torch.tensor([float(rank + 1)])
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    q.put((rank, t.tolist(), tm.item()))
    dist.destroy_process_group()


def test_gloo_two_ranks_own_each_basis_once():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=120)
    for rank, t, tm in out:
        assert t == [1.0] * 27
        assert tm == 2.0

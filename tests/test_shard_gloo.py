"""Multi-rank host logic on CPU: two gloo ranks shard an uneven batch with
partition(), each 'inverts' its share (here: records its indices and a cheap
checksum computed on the host), and the gather covers every matrix exactly
once with balanced n^3 loads.  No GPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2208_01239_gb300 import shard
from paper_2208_01239_gb300 import workloads as W


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = W.uneven_sizes(1024, 32, 512, seed=4)
    parts = shard.partition(sizes, world)
    mine = torch.tensor(parts[rank], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([len(mine)]))
    mx = max(int(c) for c in counts)
    padded = torch.full((mx,), -1, dtype=torch.int64)
    padded[: len(mine)] = mine
    gathered = [torch.zeros(mx, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(gathered, padded)
    # timing reduction as in bench.py: the slowest rank sets the time
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        allidx = torch.cat([g[g >= 0] for g in gathered]).tolist()
        q.put((sorted(allidx), shard.loads(sizes, parts), float(t.item())))
    dist.destroy_process_group()


def test_partition_single_process():
    sizes = W.uneven_sizes(1024, 32, 512, seed=4)
    parts = shard.partition(sizes, 4)
    assert sorted(i for p in parts for i in p) == list(range(1024))
    ld = shard.loads(sizes, parts)
    assert max(ld) <= 1.01 * (sum(ld) / 4) + max(int(n) ** 3 for n in sizes)
    assert shard.partition([5], 3) == [[0], [], []]


def test_two_gloo_ranks_cover_the_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    allidx, ld, tmax = q.get(timeout=60)
    assert allidx == list(range(1024))
    assert abs(ld[0] - ld[1]) <= 512 ** 3
    assert tmax == 2.0

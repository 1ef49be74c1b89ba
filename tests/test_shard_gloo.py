"""Multi-rank host logic on CPU: two gloo ranks shard an uneven batch with
partition(); the gather covers every matrix exactly once with balanced n^3
loads, and in a second test each rank inverts its share (through the CPU
oracle's Frobenius inversion, standing in for the GPU call) and rank 0 checks
every gathered inverse.  No GPU."""
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


def _invert_worker(rank, world, port, q):
    import numpy as np

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes, mats = W.uneven_batch(24, 3, 40, seed=41)
    parts = shard.partition(sizes, world)
    nmax = int(max(sizes))
    # each rank's inverses, zero-padded to nmax x nmax, as (re, im) planes
    mine = torch.zeros((len(sizes), 2, nmax, nmax), dtype=torch.float64)
    for i in parts[rank]:
        x = oracle.frob_inv_lu(mats[i])
        n = x.shape[0]
        mine[i, 0, :n, :n] = torch.from_numpy(np.ascontiguousarray(x.real))
        mine[i, 1, :n, :n] = torch.from_numpy(np.ascontiguousarray(x.imag))
    dist.all_reduce(mine)  # disjoint shares: the sum is the gather
    if rank == 0:
        worst = 0.0
        for i, n in enumerate(sizes):
            x = mine[i, 0, :n, :n].numpy() + 1j * mine[i, 1, :n, :n].numpy()
            r = mats[i] @ x - np.eye(n)
            worst = max(worst, float(np.linalg.norm(r) / (np.linalg.norm(mats[i]) * np.linalg.norm(x))))
        q.put(worst)
    dist.destroy_process_group()


def test_two_gloo_ranks_invert_their_shares():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30600 + os.getpid() % 1000
    mp.start_processes(_invert_worker, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    worst = q.get(timeout=60)
    assert worst <= 1e-13

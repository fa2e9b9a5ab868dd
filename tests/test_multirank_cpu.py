"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own seeded source
shard of one replicated graph, and bench.reduce_bc's sum all-reduce of the BC vector.

BC is additive over sources (Alg. 1 sums the dependencies of each source independently),
so the whole-job result of the ranks' shards is the sum of their per-shard vectors; the
job's time is the slowest rank's (max over ranks).  The oracle stands in for the GPU
kernels here (tests/test_gpu_multirank.py runs the library in two processes)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import bench
    import graphgen as gg
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (rank, world, rank)
    g = gg.rmat(9, 8, 1)
    src = bench.rank_sources(g, 12, rank)
    part = oracle.bc(g, src, nthreads=1)
    fake_ms = 10.0 + 5.0 * rank  # each rank's own step time
    slowest = bench.max_over_ranks(fake_ms, dist, "cpu")
    total = bench.reduce_bc(torch.from_numpy(part.copy()), dist)
    shards = [None] * world
    dist.all_gather_object(shards, src.tolist())
    if rank == 0:
        np.savez(os.path.join(out_dir, "r0.npz"), total=total.numpy(), slowest=slowest,
                 shards=np.array(shards, dtype=np.int64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_sources(tmp_path):
    world = 2
    mp.start_processes(worker, args=(world, free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    import graphgen as gg
    import oracle
    import bench
    z = np.load(tmp_path / "r0.npz")
    g = gg.rmat(9, 8, 1)
    s0, s1 = z["shards"]
    assert (s0 == bench.rank_sources(g, 12, 0)).all()
    assert set(s0.tolist()) != set(s1.tolist())  # each rank draws its own work
    assert float(z["slowest"]) == 15.0
    union = oracle.bc(g, np.concatenate([s0, s1]).astype(np.int32))
    err = np.abs(z["total"] - union) / np.maximum(np.abs(union), 1.0)
    assert err.max() <= 1e-12


def test_single_rank_needs_no_process_group():
    import torch
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    v = torch.arange(4, dtype=torch.float64)
    assert bench.reduce_bc(v, None) is v

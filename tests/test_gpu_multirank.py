"""Two processes, each with its own context on cuda:0, run the library on their own source
shards of one graph; a gloo all-reduce (bench.reduce_bc, the step of bench.py's N > 1 path)
sums their BC vectors, and the sum must equal the oracle's BC over the union of the shards.

BC is additive over sources (Alg. 1 sums each source's dependencies independently), which
is what the paper's coarse-grained multi-GPU mode rests on (Sec. 3.3 sub-clustering with one
source set per GPU).  Both processes use the per-source path on a graph of 4096 vertices,
whose kernel runs each source inside one CTA (no grid-wide waits), so the two processes'
kernels never wait on one another."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    import graphgen as gg
    import paper_1602_00963_gb300 as bc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.rmat(12, 16, 1)
    src = bench.rank_sources(g, 200, rank)
    ctx = bc.bc_ctx_create(0)
    h = bc.bc_graph_create(ctx, g.n, g.row_ptr, g.col_idx, g.nnz, bc.BC_VALIDATE)
    part, st = bc.bc_sources(h, g.n, src, bc.BC_PATH_PLAIN)
    bc.bc_destroy(h)
    bc.bc_destroy(ctx)
    total = bench.reduce_bc(torch.from_numpy(part.copy()), dist)
    shards = [None] * world
    dist.all_gather_object(shards, src.tolist())
    if rank == 0:
        np.savez(os.path.join(out_dir, "r0.npz"), total=total.numpy(),
                 shards=np.array(shards, dtype=np.int64), sources=st["sources"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_processes_shard_sources_and_sum_bc(tmp_path):
    import torch.multiprocessing as mp
    import graphgen as gg
    import oracle
    from bcgpu import assert_bc_close
    world = 2
    mp.start_processes(worker, args=(world, free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    z = np.load(tmp_path / "r0.npz")
    s0, s1 = z["shards"]
    assert set(s0.tolist()) != set(s1.tolist())
    assert int(z["sources"]) == s0.size
    g = gg.rmat(12, 16, 1)
    want = oracle.bc(g, np.concatenate([s0, s1]).astype(np.int32))
    assert_bc_close(z["total"], want, what="sum of two processes' shards vs the oracle on the union")

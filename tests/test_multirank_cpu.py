"""The benchmark's multi-rank host logic on two CPU ranks (gloo, 127.0.0.1):
every rank gets its own run seeds, the job time is the slowest rank's, and
the whole-job rate counts all ranks' work (weak scaling, no collective on the
data path)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.rank_seed(1002, rank)
    local_seconds = 1.0 + rank  # rank 1 is the slow one
    t = bench.max_over_ranks(local_seconds, world, "cpu")
    rate = bench.whole_job_rate(50_000, world, t)
    seeds = [None] * world
    dist.all_gather_object(seeds, seed)
    out[rank] = (t, rate, tuple(seeds))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    (t0, r0, s0), (t1, r1, s1) = out[0], out[1]
    assert t0 == t1 == 2.0                      # the slowest rank's time
    assert r0 == r1 == 2 * 50_000 / 2.0         # all ranks' units over it
    assert s0 == s1 and len(set(s0)) == 2       # distinct ensembles per rank

"""The ensemble-sharded solve's host logic on two CPU ranks (gloo, 127.0.0.1).

Algorithm 2 runs once over a global ensemble whose runs are split into
contiguous blocks, one per rank: every rank must see all fits and coherences
in global order and pick the same run as the oracle's rule applied to the
concatenation, including at the inclusive 1.05 boundary and on coherence
ties (lowest global index).  The benchmark's job time is the slowest rank's,
and its rate counts all ranks' work (weak scaling)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import build, sharded


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _global_ensemble(total, case):
    rng = np.random.default_rng(100 + case)
    fit = rng.uniform(10.0, 11.0, total)
    mu = rng.uniform(0.0, 1.0, total)
    if case == 1:  # a run exactly at the inclusive threshold with the lowest coherence, on the other rank
        fit[:] = rng.uniform(10.6, 11.0, total)
        fit[2] = 10.0
        fit[total - 1] = 10.0 * 1.05
        mu[total - 1] = -1.0
    if case == 2:  # equal coherences across the rank boundary: the lowest global index wins
        fit[:] = 10.0
        mu[:] = 0.5
    if case == 3:  # non-finite fits are excluded
        fit[0] = np.nan
        fit[total - 2] = np.inf
    return fit, mu


def test_shard_bounds_partition_every_run_once():
    for total in (0, 1, 7, 50, 64, 129):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = sharded.shard_bounds(total, r, world)
                seen += list(range(lo, hi))
                assert hi - lo in (total // world, total // world + 1)
                assert all(sharded.owner_of(m, total, world) == r for m in range(lo, hi))
            assert seen == list(range(total))
    with pytest.raises(ValueError):
        sharded.shard_bounds(10, 2, 2)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for case in range(4):
        total = 13  # uneven blocks: 7 + 6
        fit, mu = _global_ensemble(total, case)
        lo, hi = sharded.shard_bounds(total, rank, world)
        best, gfit, gmu = sharded.global_select(fit[lo:hi], mu[lo:hi])  # the library's host rule
        res[case] = (best, gfit.tolist(), gmu.tolist())
    t = bench.max_over_ranks(1.0 + rank, world, "cpu")
    res["time"] = (t, bench.whole_job_rate(50_000, world, t))
    out[rank] = res
    dist.destroy_process_group()


def test_two_rank_global_selection_gloo():
    build.build_library()  # the selection rule is the library's host code
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
    assert all(p.exitcode == 0 for p in procs)
    for case in range(4):
        fit, mu = _global_ensemble(13, case)
        want = O.select(fit, mu)
        for r in range(2):
            best, gfit, gmu = out[r][case]
            assert best == want, (case, r, best, want)
            assert np.array_equal(np.asarray(gfit), fit, equal_nan=True) and np.array_equal(gmu, mu)
    assert O.select(*_global_ensemble(13, 1)) == 12   # the boundary run on rank 1 wins
    assert O.select(*_global_ensemble(13, 2)) == 0    # tie: lowest global index
    (t0, r0), (t1, r1) = out[0]["time"], out[1]["time"]
    assert t0 == t1 == 2.0                   # the slowest rank's time
    assert r0 == r1 == 2 * 50_000 / 2.0      # all ranks' units over it

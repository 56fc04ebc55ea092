"""Ensemble sharding across GPUs (one process per GPU).

The M runs of Algorithm 2 are independent until the selection: each run of
Algorithm 1 touches only the shared data X and its own A and B (Sec. III-D).
So a world*M-run ensemble splits into contiguous blocks of runs, one block
per rank, with X replicated; no data moves between ranks during the solve.
The one exchange step is Algorithm 2 itself: it needs every run's fit and
coherence.  Each rank contributes its 2 M doubles to one all-gather, and
every rank applies the selection rule (the library's own edaa_select_rule)
to the concatenation, so all ranks agree on the selected run and on the rank
that holds it.

The alternative split -- pixels across ranks, with an all-reduce of the
per-pass partial sums (X W, the softmax denominators and maxima) after every
pass -- is not built: it moves about 2 L M p doubles per pass instead of 2 M
doubles per solve.
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

import numpy as np


def shard_bounds(total_runs: int, rank: int, world: int) -> Tuple[int, int]:
    """Half-open range [lo, hi) of the global run indices that rank `rank` of
    `world` solves: contiguous blocks whose sizes differ by at most one, the
    larger blocks first."""
    if world < 1 or not 0 <= rank < world or total_runs < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, total_runs >= 0")
    base, extra = divmod(total_runs, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def owner_of(run: int, total_runs: int, world: int) -> int:
    """Rank that holds global run `run`."""
    for r in range(world):
        lo, hi = shard_bounds(total_runs, r, world)
        if lo <= run < hi:
            return r
    raise ValueError("run index out of range")


def gather_runs(values: Sequence[float], group=None) -> np.ndarray:
    """All ranks' per-run values (FP64) in global run order; blocks may differ
    in length by one (shard_bounds), so lengths are gathered first."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    local = torch.as_tensor(np.asarray(values, np.float64), device=dev)
    n = torch.tensor([local.numel()], dtype=torch.int64, device=dev)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    width = int(max(int(x.item()) for x in ns))
    padded = torch.full((width,), float("nan"), dtype=torch.float64, device=dev)
    padded[:local.numel()] = local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return np.concatenate([p[:int(k.item())].cpu().numpy() for p, k in zip(parts, ns)])


def global_select(fit_local: Sequence[float], mu_local: Sequence[float], ratio: float = 1.05,
                  group=None, rule=None) -> Tuple[int, np.ndarray, np.ndarray]:
    """Algorithm 2 over the whole sharded ensemble: I = {m : fit_m <= ratio *
    min fit}, best = argmin over I of mu_m, ties to the lowest global index,
    non-finite fits excluded.  Returns (best global index or -1, all fits,
    all coherences).  `rule` defaults to the library's edaa_select_rule."""
    fit = gather_runs(fit_local, group)
    mu = gather_runs(mu_local, group)
    if rule is None:
        from paper_2209_11002_gb300 import edaa
        rule = edaa.select_rule
    return int(rule(fit, mu, ratio)), fit, mu

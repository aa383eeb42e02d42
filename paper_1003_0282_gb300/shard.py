"""Distribution of a batch of independent domains over ranks (one GPU each).

The domains of a batch are independent problems, so ranks exchange nothing
on the data path: each advances its own domains with one persistent launch
per step.  Two ways to fill the ranks:

* ``weak``: every rank advances a sweep of its own (seed + rank), so the
  work per GPU stays fixed as the number of GPUs grows;
* ``strong``: one sweep is split into disjoint subsets with balanced node
  counts (largest domain first onto the least-loaded rank).

Host-side helpers gather per-domain results on every rank and take the
slowest rank's time.  They run over any ``torch.distributed`` backend
(NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def balanced_shards(cells: Sequence[int], world: int) -> List[List[int]]:
    """Indices of the domains each rank gets: disjoint, covering, and with
    node counts that differ by at most the largest domain (greedy LPT;
    deterministic: ties go to the lower rank, equal domains by index).
    Each rank's list is in increasing domain order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for d in sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(d)
        load[r] += int(cells[d])
    return [sorted(x) for x in out]


def rank_problems(sweep, world: int, rank: int, mode: str = "weak", seed: int = 20261202, **kw):
    """The problems rank ``rank`` of ``world`` advances.  ``sweep`` is a
    function (seed=..., **kw) -> list of problems (e.g. inputs.batch_sweep)."""
    if mode == "weak":
        return sweep(seed=seed + rank, **kw)
    if mode == "strong":
        full = sweep(seed=seed, **kw)
        shards = balanced_shards([p.cells for p in full], world)
        return [full[d] for d in shards[rank]]
    raise ValueError(f"unknown sharding mode {mode!r}")


def _device_for(dist):
    import torch
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def max_over_ranks(value: float) -> float:
    """The largest of the ranks' values (every rank gets it)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device_for(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float) -> float:
    """The sum of the ranks' values (every rank gets it)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device_for(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_per_domain(local: np.ndarray, shard: Sequence[int], n_total: int) -> np.ndarray:
    """Assemble per-domain rows (e.g. residual, mass, budget) that each rank
    computed for its shard into one [n_total, k] array on every rank."""
    import torch.distributed as dist
    local = np.asarray(local, dtype=np.float64)
    if local.shape[0] != len(shard):
        raise ValueError("one row per domain of the shard")
    if not dist.is_initialized() or dist.get_world_size() == 1:
        parts = [(list(shard), local)]
    else:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, (list(shard), local))
    out = np.full((n_total, local.shape[1]), np.nan)
    seen = np.zeros(n_total, dtype=bool)
    for idx, rows in parts:
        for i, d in enumerate(idx):
            if seen[d]:
                raise ValueError(f"domain {d} appears on two ranks")
            seen[d] = True
            out[d] = rows[i]
    if not seen.all():
        raise ValueError("some domains are on no rank")
    return out

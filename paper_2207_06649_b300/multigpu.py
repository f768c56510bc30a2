"""Multi-GPU host logic.  Environments are independent (Sec. IV-C runs N_e separate
environments), so the rollout path shards with no exchange between GPUs: either each
rank runs its own workload (weak scaling, the benchmark's mode) or one batch is split
into contiguous environment ranges balanced by box count, with a host gather of the
per-environment results.  The only collective is the timing reduction of the benchmark
(maximum time over ranks, summed work)."""
from __future__ import annotations

import numpy as np


def rank_seed(base_seed: int, rank: int) -> int:
    """Workload seed of a rank in weak scaling: every rank simulates its own scenes."""
    return base_seed + 1000 * rank


def partition_envs(box_counts, world: int):
    """Split environments 0..E-1 into `world` contiguous ranges whose box totals (the
    work of a rollout grows with the box count) are as even as a prefix split allows.
    Returns offsets [world + 1]."""
    w = np.asarray(box_counts, np.float64)
    E = len(w)
    if world <= 1 or E == 0:
        return np.array([0, E], np.int64) if world <= 1 else np.zeros(world + 1, np.int64)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    off = [0]
    for r in range(1, world):
        goal = total * r / world
        k = int(np.searchsorted(cum, goal))
        # take the nearer boundary of the two around the goal, keeping ranges ordered
        if k > 0 and abs(cum[k - 1] - goal) <= abs(cum[min(k, E)] - goal):
            k -= 1
        off.append(max(off[-1], min(k, E)))
    off.append(E)
    return np.array(off, np.int64)


def reduce_job(elapsed_s: float, work: float, device=None):
    """(max elapsed over ranks, summed work) with torch.distributed; identity when not
    initialised.  device: where the reduction tensor lives (CUDA for NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s), float(work)
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    return float(t.item()), float(s.item())

"""Multi-GPU host logic: instances are independent (each is its own evolution), so a batch is
split across ranks with no collective on the data path -- one process per GPU, each running its
own solver on its share.  The only exchanges are host-side: the per-instance results gathered
to rank 0 once at the end, and the timing reduction (max over ranks) of a benchmark.

partition(): longest-processing-time-first assignment of instances to ranks by estimated work
(N times RK4 steps to t_end, i.e. grid points times steps), which keeps the ranks within one
instance's work of each other.
"""
from __future__ import annotations

import math

import numpy as np


def instance_work(N, t_end, cfl=0.5, cadence=1.0):
    """Estimated work of each instance: N times its RK4 step count to t_end (the library's
    dt = cadence / ceil(cadence / (cfl h)), h = pi / (2 (N - 1)))."""
    N = np.asarray(N, dtype=np.int64)
    h = 0.5 * math.pi / (N - 1)
    dt = cadence / np.ceil(cadence / (cfl * h))
    return N * np.ceil(t_end / dt - 1e-9)


def partition(work, world):
    """Indices of the instances of every rank: largest work first, each to the least-loaded
    rank (ties to the lowest rank); every rank's list is in increasing index order."""
    work = np.asarray(work, dtype=np.float64)
    load = np.zeros(world)
    parts = [[] for _ in range(world)]
    for i in sorted(range(work.size), key=lambda k: (-work[k], k)):
        r = int(np.argmin(load))
        parts[r].append(i)
        load[r] += work[i]
    return [sorted(p) for p in parts]


def gather_results(local, indices, B, dist, dtype=np.float64, group=None):
    """Reassemble per-instance results (local: array of this rank's instances, in the order of
    `indices`) into the global order on rank 0 (None elsewhere).  Host tensors over `group`
    (default: the default process group), which must have a host backend (gloo)."""
    import torch
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    payload = np.concatenate([np.asarray(indices, dtype=np.float64)[:, None],
                              np.asarray(local, dtype=np.float64).reshape(len(indices), -1)], axis=1)
    width = payload.shape[1]
    counts = torch.zeros(world, dtype=torch.int64)
    counts[rank] = len(indices)
    dist.all_reduce(counts, group=group)
    nmax = int(counts.max())
    buf = torch.zeros((nmax, width), dtype=torch.float64)
    buf[: len(indices)] = torch.from_numpy(payload)
    out = [torch.zeros_like(buf) for _ in range(world)] if rank == 0 else None
    dist.gather(buf, out, dst=0, group=group)
    if rank != 0:
        return None
    res = np.zeros((B, width - 1))
    for r in range(world):
        rows = out[r][: int(counts[r])].numpy()
        res[rows[:, 0].astype(np.int64)] = rows[:, 1:]
    res = res.astype(dtype)
    return res[:, 0] if width == 2 else res


def reduce_timing(seconds, work, dist, device=None):
    """(max seconds over ranks, total work over ranks): the whole-job rate is work / seconds."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())

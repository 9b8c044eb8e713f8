"""Running one trajectory ensemble on several GPUs (one process per GPU).

Trajectories are independent (the paper's Sec. 3.2: the computation is embarrassingly parallel), so
the only multi-GPU pieces are (i) giving each rank a disjoint set of trajectory ids -- the Philox key
is the trajectory id, so results do not depend on the partition -- and (ii) one reduction at the end
of (sum S, sum S^2, count) per observable and group, from which the ensemble means and their
standard errors follow.  There is no exchange on the hot path.
"""
from __future__ import annotations

import numpy as np


def shard(n_total: int, rank: int, world: int) -> np.ndarray:
    """Contiguous, disjoint, near-equal blocks of trajectory ids for each rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return np.arange(start, start + base + (1 if rank < extra else 0), dtype=np.int64)


def local_moments(obs: np.ndarray, group: np.ndarray, n_groups: int) -> np.ndarray:
    """(n_groups, 3, NBASIS) array of (sum S, sum S^2, count) of the survival ratios per group."""
    surv = obs["surv"]
    out = np.zeros((n_groups, 3, surv.shape[1]), dtype=np.float64)
    for g in range(n_groups):
        s = surv[group == g]
        out[g, 0] = s.sum(axis=0)
        out[g, 1] = (s * s).sum(axis=0)
        out[g, 2] = len(s)
    return out


def reduce_moments(m: np.ndarray) -> np.ndarray:
    """Sums the moments over all ranks of the default torch.distributed group (a no-op when it is
    not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return m
    t = torch.from_numpy(np.ascontiguousarray(m))
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def ensemble(m: np.ndarray):
    """Means and standard errors of the mean from the reduced moments."""
    n = np.maximum(m[:, 2], 1.0)
    mean = m[:, 0] / n
    var = np.maximum(m[:, 1] / n - mean * mean, 0.0)
    return mean, np.sqrt(var / np.maximum(n - 1.0, 1.0))

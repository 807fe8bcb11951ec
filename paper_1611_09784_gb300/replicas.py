"""Replica (one process per GPU) merging of MLMC level accumulators.

The samples of different ranks are independent (disjoint seeds or sample
ranges), so replicas exchange only the per-level float64 accumulators
(M_l, sum Y, sum Y^2) once, with a sum over ranks; the eq. (2.6) combine of
the merged sums is the library's idos_combine_level_stats.  Works with any
torch.distributed backend (gloo on CPU, NCCL on GPU).
"""
from __future__ import annotations

import numpy as np


def model_stats(model):
    """(counts int64[L], sums float64[L, 2, n_E]) of a Model's accumulators."""
    L = model.n_levels
    counts = np.zeros(L, dtype=np.int64)
    sums = np.zeros((L, 2, model.n_E))
    for l in range(L):
        M, s1, s2, _ = model.get_level_stats(l)
        counts[l] = M
        sums[l, 0] = s1
        sums[l, 1] = s2
    return counts, sums


def merge(counts, sums, group=None, device=None):
    """Sum the accumulators over all ranks of `group` (torch.distributed)."""
    import torch
    import torch.distributed as dist
    c = torch.as_tensor(np.asarray(counts, dtype=np.float64), device=device)
    s = torch.as_tensor(np.asarray(sums, dtype=np.float64), device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    return c.cpu().numpy().round().astype(np.int64), s.cpu().numpy()


def combine(counts, sums):
    """Eq. (2.6) estimate and its variance from merged accumulators
    (idos_combine_level_stats)."""
    from .binding import combine_level_stats
    return combine_level_stats(counts, sums)

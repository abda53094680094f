"""Initial states spread over ranks (the paper's first level of parallelism,
Sec. V): each rank integrates a subset of the initial conditions, and one
sum-reduction of (G, dG/dalpha) over ranks gives the full objective and
gradient.

G = 1/M sum_i beta_i J_i + gamma2/2 ||alpha||^2 splits exactly: rank r holds
the states I_r and reports G_r = 1/M sum_{i in I_r} beta_i J_i (+ the Tikhonov
term on rank 0 only).  A local solve over M_r states divides by M_r, so the
rank's weights become beta_i M_r / M.
"""

from __future__ import annotations

import copy

import numpy as np


def shard_indices(M: int, rank: int, world: int) -> np.ndarray:
    """States of ``rank``: a contiguous, balanced block of range(M)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(M, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return np.arange(start, stop)


def shard_problem(prob, rank: int, world: int):
    """The sub-problem of ``rank`` (None when it holds no state): its states,
    targets and gate objective, weights rescaled by M_r/M, and the Tikhonov
    term kept on rank 0 only."""
    idx = shard_indices(prob.M, rank, world)
    if idx.size == 0:
        return None
    sub = copy.deepcopy(prob)
    sub.rho0 = np.asarray(prob.rho0)[idx]
    if prob.targets is not None:
        sub.targets = np.asarray(prob.targets)[idx]
    w = np.ones(prob.M) if prob.weights is None else np.asarray(prob.weights, dtype=np.float64)
    sub.weights = w[idx] * (idx.size / prob.M)
    if rank != 0:
        sub.gamma2 = 0.0
    return sub


def allreduce_objective(G: float, grad: np.ndarray, group=None):
    """Sum (G, grad) over the ranks of ``group`` (torch.distributed); returns
    the totals on every rank."""
    import torch
    import torch.distributed as dist

    buf = torch.from_numpy(np.concatenate([[G], np.asarray(grad, dtype=np.float64)]))
    if dist.get_backend(group) == "nccl":
        buf = buf.cuda()
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    out = buf.cpu().numpy()
    return float(out[0]), out[1:]

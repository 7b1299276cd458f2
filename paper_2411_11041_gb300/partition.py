"""Splitting a batch of independent problems over GPUs (one process per GPU).

The problems of a batch share nothing, so N ranks solve disjoint subsets with
no exchange step: each rank runs its own batched solve, and only results and
timings cross ranks.  The subsets are chosen by longest processing time first
(LPT) on an estimate of each problem's work, so that the slowest rank, which
sets the job's time, carries as little as possible.  Every rank computes the
same split from the same problem list (the rule is deterministic).
"""
from __future__ import annotations

import math

import numpy as np


def work_estimate(prob) -> float:
    """Line unknowns per split step times the expected number of split steps.

    The unknowns are about the active nodes of each of the two families.  With
    the default pseudo step dt = 2 / sqrt(lmin lmax) the split iteration
    contracts like a Peaceman-Rachford step, so its step count grows like
    sqrt(lmax / lmin), lmin = sigma, lmax = 12 mu / h^2 + 2 sqrt(3) max|beta| / h."""
    h = min((prob.x1 - prob.x0) / (prob.nx - 1), (prob.y1 - prob.y0) / (prob.ny - 1))
    mask = np.asarray(prob.mask) != 0
    b = np.hypot(np.asarray(prob.beta1), np.asarray(prob.beta2))
    bmax = float(b[mask].max()) if mask.any() else 0.0
    lmax = 12.0 * prob.mu / (h * h) + 2.0 * math.sqrt(3.0) * bmax / h
    return 2.0 * float(mask.sum()) * math.sqrt(lmax / prob.sigma)


def lpt_split(works, n_ranks: int):
    """Problem indices of each rank and the ranks' estimated loads: problems
    longest first, each to the least-loaded rank (ties to the lower rank and
    the lower index).  The largest load is within 4/3 of the best split's."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(works)), key=lambda i: (-float(works[i]), i))
    loads = [0.0] * n_ranks
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        r = min(range(n_ranks), key=lambda k: (loads[k], k))
        parts[r].append(i)
        loads[r] += float(works[i])
    return [sorted(p) for p in parts], loads

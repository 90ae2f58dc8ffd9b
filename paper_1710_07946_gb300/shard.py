"""Host-side partition of one batch of independent blocks across GPUs.

The generators of the neutered block columns of an HSS / FMM matrix are
independent low-rank approximations (paper: Section "Application: HSS / FMM",
stage (ii)), so a batch shards with no exchange on the data path: every rank
runs the C-A batch of its share, and the ranks meet once afterwards to add
their counts.  The share is chosen by the longest-processing-time-first rule
(Graham's LPT list scheduling) on a per-block cost such as rows x columns x k:
blocks in order of decreasing cost, each given to the rank with the smallest
load so far.
"""
from __future__ import annotations

import numpy as np


def lpt_partition(costs, nparts: int):
    """Indices of the blocks of each of ``nparts`` parts under LPT list
    scheduling of ``costs`` (one non-negative number per block).

    Blocks are taken in decreasing cost (ties: lower index first) and each goes
    to the part with the least total cost so far (ties: lower part).  Every block
    lands in exactly one part; each part's indices are returned in ascending
    order.  The loads of any two parts differ by at most the largest cost."""
    costs = np.asarray(costs, dtype=np.float64).reshape(-1)
    if nparts < 1:
        raise ValueError("nparts >= 1")
    if np.any(costs < 0) or not np.all(np.isfinite(costs)):
        raise ValueError("costs must be finite and non-negative")
    order = np.lexsort((np.arange(len(costs)), -costs))
    load = np.zeros(nparts)
    owner = np.empty(len(costs), dtype=np.int64)
    for b in order:
        r = int(np.argmin(load))                     # first minimum: the lowest part on ties
        owner[b] = r
        load[r] += costs[b]
    return [np.flatnonzero(owner == r) for r in range(nparts)]


def block_costs(blocks, k: int):
    """rows x columns x min(k, rows, columns) per block (blocks: nb x 4 of
    row0, nrows, col0, ncols): the size of a block's C-A work."""
    b = np.asarray(blocks, dtype=np.int64).reshape(-1, 4)
    kb = np.minimum(k, np.minimum(b[:, 1], b[:, 3]))
    return (b[:, 1] * b[:, 3] * kb).astype(np.float64)

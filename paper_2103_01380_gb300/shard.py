"""Sharding subdomains across GPUs (one process per GPU).

Subdomains are independent -- the ID needs no communication between blocks
(Section 3.2) -- so ranks share nothing on the data path.  Each rank takes a
subset of subdomains chosen by longest-processing-time-first on m_s n_s (the
bytes each one streams), and the only exchange is one host-side sum of four
doubles per window: sum ||E||_F^2, sum ||A||_F^2, sum m n and sum k (m + n),
from which the global relative error (Section 5.1) and the aggregate
compression factor (Section 2, Eq. for CF) follow.
"""
from __future__ import annotations

import heapq

import numpy as np


def lpt_partition(weights, nranks: int):
    """Assign items to ranks, heaviest first onto the least-loaded rank.

    Returns a list of sorted index arrays, one per rank (deterministic: ties
    go to the lower item index and the lower rank)."""
    w = np.asarray(weights, dtype=np.float64)
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    heap = [(0.0, r) for r in range(nranks)]
    heapq.heapify(heap)
    parts = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + w[i], r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def combine_totals(totals, group=None):
    """Sum the per-rank [sum e2, sum a2, sum mn, sum k(m+n)] over the process
    group (a gloo group on host tensors) and return (relative error, CF,
    the summed four-vector)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(totals, dtype=np.float64).reshape(4)).clone()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    v = t.numpy()
    rel = float(np.sqrt(v[0] / v[1])) if v[1] > 0 else 0.0
    cf = float(v[2] / v[3]) if v[3] > 0 else float("inf")
    return rel, cf, v

"""Sharding subdomains across GPUs (one process per GPU).

Subdomains are independent -- the ID needs no communication between blocks
(Section 3.2) -- so ranks share nothing on the data path.  Each rank takes a
subset of subdomains chosen by longest-processing-time-first on m_s n_s (the
bytes each one streams), and the only exchange is one host-side sum per
window of sum ||E||_F^2, sum ||A||_F^2, sum m n and sum k (m + n) (plus the
per-QoI sums of ||E||^2 and ||A||^2 when subdomains hold one QoI each), from
which the global and per-QoI relative errors (Section 5.1) and the aggregate
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


def domain_boxes(world: int, boxes_per_domain: int, weight: float = 1.0):
    """The subdomain set of a run on `world` ranks: one domain of
    boxes_per_domain boxes per rank (so each GPU's share stays fixed as ranks
    are added), every (domain, box) unit of weight m n, dealt by lpt_partition.
    Returns, per rank, an array of (domain, box) pairs."""
    units = world * boxes_per_domain
    parts = lpt_partition(np.full(units, float(weight)), world)
    return [np.stack([p // boxes_per_domain, p % boxes_per_domain], axis=1) for p in parts]


def combine_totals(totals, group=None):
    """Sum the per-rank [sum e2, sum a2, sum mn, sum k(m+n), (e2_q, a2_q) per
    QoI ...] over the process group (a gloo group on host tensors) and return
    (relative error, CF, the summed vector)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(totals, dtype=np.float64).reshape(-1)).clone()
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    v = t.numpy()
    rel = float(np.sqrt(v[0] / v[1])) if v[1] > 0 else 0.0
    cf = float(v[2] / v[3]) if v[3] > 0 else float("inf")
    return rel, cf, v


def per_qoi_rel_err(v) -> np.ndarray:
    """sqrt(e2_q / a2_q) from a summed totals vector with per-QoI pairs."""
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    g = v[4:].reshape(-1, 2)
    return np.sqrt(g[:, 0] / g[:, 1])

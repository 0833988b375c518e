"""Multi-rank host logic on CPU: LPT sharding of subdomains and the one
four-double reduction across ranks (gloo, world size 2).  The device path is
unchanged per rank; this covers what crosses ranks."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2103_01380_gb300 import shard


def test_lpt_partition_is_balanced_and_complete():
    rng = np.random.default_rng(4)
    edges = rng.choice([8, 12, 16, 24, 32], size=300)
    n = rng.integers(64, 1025, size=300)
    w = 5 * edges ** 3 * n
    parts = shard.lpt_partition(w, 4)
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(300))
    loads = [w[p].sum() for p in parts]
    # LPT bound: max load <= 4/3 optimum (and the optimum >= mean)
    assert max(loads) <= (4.0 / 3.0) * max(np.mean(loads), w.max())
    assert shard.lpt_partition(w, 4)[0].tolist() == parts[0].tolist()   # deterministic


def test_single_rank_totals_without_a_group():
    rel, cf, v = shard.combine_totals([1.0, 4.0, 400 * 100, 500])
    assert rel == pytest.approx(0.5)
    assert cf == pytest.approx(80.0)     # Section 5.1 case: 400 x 100 at rank 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # every rank compresses its LPT share with the oracle and reports its sums
        rng = np.random.default_rng(11)
        blocks = [rng.standard_normal((60 + 10 * s, 3)) @ rng.standard_normal((3, 20 + s))
                  + 1e-3 * rng.standard_normal((60 + 10 * s, 20 + s)) for s in range(6)]
        weights = [b.size for b in blocks]
        mine = shard.lpt_partition(weights, world)[rank]
        tot = np.zeros(4)
        for s in mine:
            r = oracle.spid(blocks[s], 8, 3, 0.0, 2.0 ** -53, 5)
            m, n = blocks[s].shape
            tot += [r["e2"], r["a2"], m * n, r["k"] * (m + n)]
        rel, cf, v = shard.combine_totals(tot)
        q.put((rank, rel, cf, list(v)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_totals():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the same window on one rank
    rng = np.random.default_rng(11)
    blocks = [rng.standard_normal((60 + 10 * s, 3)) @ rng.standard_normal((3, 20 + s))
              + 1e-3 * rng.standard_normal((60 + 10 * s, 20 + s)) for s in range(6)]
    tot = np.zeros(4)
    for b in blocks:
        r = oracle.spid(b, 8, 3, 0.0, 2.0 ** -53, 5)
        tot += [r["e2"], r["a2"], b.size, r["k"] * sum(b.shape)]
    rel1, cf1, _ = shard.combine_totals(tot)
    for rank, rel, cf, v in out:
        assert rel == pytest.approx(rel1, rel=1e-12)
        assert cf == pytest.approx(cf1, rel=1e-12)


def _dead_peer_worker(rank, world, port, q):
    import datetime
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(0)            # this rank dies between steps, before the reduction
    try:
        shard.combine_totals([1.0, 2.0, 3.0, 4.0])
        q.put("no error")
    except Exception as exc:   # the survivor gets an error, not a hang
        q.put(type(exc).__name__)


def test_a_dead_rank_gives_an_error_not_a_hang():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dead_peer_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert res != "no error"

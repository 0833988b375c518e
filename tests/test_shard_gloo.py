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


def test_domain_boxes_deals_every_box_once_and_evenly():
    # the bench's multi-GPU set: one domain of boxes per rank, (domain, box)
    # units of equal weight dealt by LPT -- each rank gets one domain's worth
    for world in (1, 2, 3, 8):
        parts = shard.domain_boxes(world, 512, weight=5 * 32 ** 3 * 256)
        units = np.sort(np.concatenate([p[:, 0] * 512 + p[:, 1] for p in parts]))
        assert np.array_equal(units, np.arange(world * 512))
        assert all(len(p) == 512 for p in parts)
        assert np.all(np.concatenate(parts)[:, 0] < world)
    assert shard.domain_boxes(1, 64)[0].tolist() == [[0, b] for b in range(64)]


def _qoi_blocks(nbox, nq=3):
    rng = np.random.default_rng(21)
    out = {}
    for d in range(2):
        for b in range(nbox):
            base = rng.standard_normal((40, 4)) @ rng.standard_normal((4, 30))
            out[(d, b)] = [(2.0 ** q) * base + 1e-3 * rng.standard_normal((40, 30))
                           for q in range(nq)]
    return out


def _qoi_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        blocks = _qoi_blocks(4)
        tot = np.zeros(4 + 2 * 3)
        for d, b in shard.domain_boxes(world, 4)[rank]:
            for qq, A in enumerate(blocks[(int(d), int(b))]):
                r = oracle.spid(A, 8, 3, 0.0, 2.0 ** -53, 5)
                tot[:4] += [r["e2"], r["a2"], A.size, r["k"] * sum(A.shape)]
                tot[4 + 2 * qq] += r["e2"]
                tot[5 + 2 * qq] += r["a2"]
        rel, cf, v = shard.combine_totals(tot)
        q.put((rank, rel, cf, list(shard.per_qoi_rel_err(v))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_per_qoi_totals():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_qoi_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    blocks = _qoi_blocks(4)
    e2 = np.zeros(3)
    a2 = np.zeros(3)
    for key in sorted(blocks):
        for qq, A in enumerate(blocks[key]):
            r = oracle.spid(A, 8, 3, 0.0, 2.0 ** -53, 5)
            e2[qq] += r["e2"]
            a2[qq] += r["a2"]
    want = np.sqrt(e2 / a2)
    for rank, rel, cf, pq in out:
        assert np.allclose(pq, want, rtol=1e-12)

"""Multi-rank host logic on CPU: two gloo ranks split a batch of independent
graphs, each solves its share (with the CPU oracle standing in for a GPU),
and the union of their results equals solving the whole batch."""
import os
import socket

import numpy as np
import pytest

import graphgen
import oracle
from paper_1910_05971_gb300.replicas import batch_work, max_over_ranks, shard_graphs, sum_over_ranks


def test_shard_graphs_is_balanced_and_deterministic():
    sizes = np.random.default_rng(0).integers(1, 10_000, size=500)
    a = shard_graphs(sizes, 4)
    assert a == shard_graphs(sizes, 4)
    assert sorted(i for r in a for i in r) == list(range(500))
    loads = [int(sizes[r].sum()) for r in a]
    assert max(loads) - min(loads) <= int(sizes.max())
    assert shard_graphs([], 3) == [[], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch = graphgen.er_batch(24, seed=31, nmax=3000)
        share = shard_graphs(batch_work(batch), world)
        mine = {}
        for g in share[rank]:
            rp, ci = batch.graph(g)
            f, it, conv, _ = oracle.fastsv(rp, ci)
            mine[g] = (f.tolist(), it)
        gathered = [None] * world
        dist.all_gather_object(gathered, (share, mine))
        t = max_over_ranks(1.0 + rank, dist)
        total = sum_over_ranks(len(share[rank]), dist)
        q.put((rank, gathered, t, total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_a_batch():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    batch = graphgen.er_batch(24, seed=31, nmax=3000)
    for rank, gathered, t, total in results:
        assert t == 2.0 and total == 24
        shares = [g[0] for g in gathered]
        assert shares[0] == shares[1]                     # same split on every rank
        merged = {}
        for _, mine in gathered:
            assert not (set(mine) & set(merged))          # no graph solved twice
            merged.update(mine)
        assert sorted(merged) == list(range(24))
        for g, (f, it) in merged.items():
            rp, ci = batch.graph(g)
            assert f == oracle.uf(rp, ci).tolist()

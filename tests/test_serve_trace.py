"""Serving workload parity: a prefix of the request trace (Poisson arrivals at
2000/s, undirected edge targets log-uniform in [1e3, 5e7], half R-MAT with
edge factor 8-32, half lattices with keep probability in [0.4, 0.9], seed 5)
replayed through the continuous-batching server at its arrival times.  The
prefix holds multi-million-vertex R-MAT and lattice requests (more than 10^7
undirected edges each) among small ones; an HBM budget far below the prefix's
total keeps requests waiting for slots, so large and small graphs share steps.
Every request's labels and iteration count must equal the CPU oracle's
(Algorithm 2; labels also against union-find), bit for bit.
"""
import threading
import time

import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu

PREFIX = 64


def _prefix():
    tr = graphgen.trace(PREFIX, seed=5)
    graphs = []
    for i in range(PREFIX):
        rp, ci = graphgen.trace_graph(tr, i)
        graphs.append((rp.astype(np.int32), np.ascontiguousarray(ci, dtype=np.int32)))
    return tr, graphs


def test_trace_prefix_through_server_matches_oracle():
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300.serve import PoolBackend, Server

    tr, graphs = _prefix()
    kinds = tr["kind"]
    und = np.array([len(ci) // 2 for _, ci in graphs])
    # the prefix reaches the trace's large sizes in both families
    assert any(und[i] > 10_000_000 for i in range(PREFIX) if kinds[i] == 0)
    assert any(und[i] > 10_000_000 for i in range(PREFIX) if kinds[i] == 1)
    assert (und < 100_000).sum() >= 10
    ref = []
    for rp, ci in graphs:
        f, it, conv, _ = oracle.fastsv(rp, ci, form="omp")
        assert conv
        ref.append((f, it))

    usage = []

    class RecordingPool(PoolBackend):
        """Pool that records how many graphs each step advances."""

        def step(self, iters):
            super().step(iters)
            st, slots, _ = fsv.fastsv_pool_usage(self.h)
            usage.append(slots)

    budget = 5 << 28  # 1.25 GiB: the largest request (about 0.54 GB) fits, the prefix (3.9 GB) does not
    total = sum(fsv.fastsv_pool_bytes(len(rp) - 1, len(ci)) for rp, ci in graphs)
    assert total > 2 * budget  # admissions must wait for harvests
    srv = Server(backend=RecordingPool(budget, 32), iters_per_step=2)
    futs = [None] * PREFIX
    arrivals = tr["t"] - tr["t"][0]
    start = time.perf_counter()

    def feeder():
        for i in range(PREFIX):
            dt = start + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            futs[i] = srv.submit(*graphs[i])

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    try:
        results = [f.result(timeout=600) for f in futs]
    finally:
        srv.close()
    for i, ((lab, it), (f, it_ref)) in enumerate(zip(results, ref)):
        assert np.array_equal(lab, f), f"request {i}: labels differ from the oracle"
        assert it == it_ref, (i, it, it_ref)
    for i in np.argsort(-und)[:4]:  # the largest requests also against union-find
        assert np.array_equal(results[i][0], oracle.uf(*graphs[i]))
    assert max(usage) >= 4  # graphs of different sizes were advanced together

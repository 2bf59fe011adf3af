"""Helpers shared by the GPU parity tests (inputs from graphgen, expected
values from the oracle only)."""
from __future__ import annotations

import functools
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import graphgen
import oracle


def torch():
    import torch as _t
    return _t


def to_dev(a, dtype=None):
    t = torch()
    x = torch().from_numpy(np.ascontiguousarray(a if dtype is None else a.astype(dtype)))
    return x.cuda()


def gpu_solve(rp, ci, bits=64, max_iters=4096, **kw):
    """Labels and stats of one graph through the C ABI (fastsv_cc)."""
    import paper_1910_05971_gb300 as fsv
    with fsv.FastSV(rowptr_bits=bits, max_iters=max_iters, **kw) as s:
        rp_d = to_dev(rp, np.int64 if bits == 64 else np.int32)
        ci_d = to_dev(ci, np.int32)
        lab = s.cc(rp_d, ci_d, check_status=False)
        st = s.stats()
        st["launches"] = s.kernel_launches()
        return lab.cpu().numpy(), st


class Solver:
    """A reusable handle for many small solves."""

    def __init__(self, bits=64, **kw):
        import paper_1910_05971_gb300 as fsv
        self.bits = bits
        self.s = fsv.FastSV(rowptr_bits=bits, **kw)

    def solve(self, rp, ci):
        rp_d = to_dev(rp, np.int64 if self.bits == 64 else np.int32)
        ci_d = to_dev(ci if len(ci) else np.zeros(1, np.int32), np.int32)
        lab = self.s.cc(rp_d, ci_d, check_status=False)
        return lab.cpu().numpy(), self.s.stats()

    def close(self):
        self.s.close()


def ragged_graphs():
    """Random graphs whose (rows + entries) land just below, on and above
    multiples of the merge-path tile, plus hubs spanning many tiles."""
    rng = np.random.default_rng(99)
    out = []
    for n, m_und in [(1, 0), (2, 1), (300, 200), (1000, 1500), (2047, 0), (2049, 1), (3000, 5000)]:
        edges = {(int(rng.integers(n)), int(rng.integers(n))) for _ in range(m_und)}
        edges = sorted({(min(u, v), max(u, v)) for u, v in edges if u != v})
        out.append(oracle.csr_from_edges(n, edges))
    # a hub adjacent to everything plus a sparse rest: one row spans many tiles
    n = 9000
    edges = [(0, i) for i in range(1, n, 2)] + [(i, i + 1) for i in range(1, n - 1, 7)]
    out.append(oracle.csr_from_edges(n, edges))
    out.append(graphgen.rmat(11, 8, seed=7, permute=True))
    out.append(graphgen.grid(50, 0.55, 33, seed=5))
    return out


def per_iteration_parity(rp, ci, bits=64, max_check=64, variant=0, **kw):
    """Compare the device pointer graph with the oracle's after every
    iteration (the device restarts with max_iters = k; the oracle steps).
    variant 1..4 selects the convergence ablation sv1..sv4."""
    import paper_1910_05971_gb300 as fsv
    n = len(rp) - 1
    f_ref = np.arange(n, dtype=np.int32)
    if variant:
        kw["variant"] = variant
    k = 0
    while True:
        k += 1
        if 1 <= variant <= 4:
            changed = oracle.sv_iteration(rp, ci, f_ref, variant)
        else:
            changed = oracle.iteration(rp, ci, f_ref)
        got, st = gpu_solve(rp, ci, bits=bits, max_iters=k, **kw)
        assert np.array_equal(got, f_ref), f"pointer graph differs after iteration {k}"
        if changed == 0:
            assert st["status"] == fsv.FASTSV_OK and st["iterations"] == k
            return k
        assert st["status"] == fsv.FASTSV_ERR_MAX_ITERS and st["iterations"] == k
        if k >= max_check:
            return k


@functools.lru_cache(maxsize=4)
def workload(name):
    return graphgen.WORKLOADS[name]()


def oracle_batch(batch, nthreads=None):
    """Per-graph oracle labels (union-find) and Algorithm 2 iteration counts."""
    G = batch.num_graphs
    labels = np.empty(int(batch.vtx_off[-1]), dtype=np.int32)
    iters = np.empty(G, dtype=np.int32)

    def one(g):
        rp, ci = batch.graph(g)
        f, it, conv, _ = oracle.fastsv(rp, ci, form="alg2")
        assert conv
        labels[batch.vtx_off[g]:batch.vtx_off[g + 1]] = f
        iters[g] = it

    with ThreadPoolExecutor(max_workers=nthreads or os.cpu_count() or 4) as ex:
        list(ex.map(one, range(G)))
    return labels, iters

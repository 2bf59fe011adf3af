"""GPU tests of the batched entry point: every graph of a batch must get the
labels and the iteration count it gets alone (its Algorithm 2 sequence
depends only on its own edges, and it stops at its own early termination)."""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from gpu_util import oracle_batch, to_dev

pytestmark = pytest.mark.gpu


def _run_batch(batch, **kw):
    import paper_1910_05971_gb300 as fsv
    with fsv.FastSV(rowptr_bits=32, **kw) as s:
        lab, iters = s.cc_batched(to_dev(batch.vtx_off), to_dev(batch.edge_off), to_dev(batch.row_ptr),
                                  to_dev(batch.col_idx if len(batch.col_idx) else np.zeros(1, np.int32)))
        st = s.stats()
        return lab.cpu().numpy(), iters.cpu().numpy(), st, s.kernel_launches()


def test_batch_of_all_small_graphs():
    graphs = []
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            graphs.append(oracle.csr_from_edges(n, [pairs[i] for i in range(len(pairs)) if mask >> i & 1]))
    batch = graphgen.Batch.from_graphs(graphs)
    lab, iters, st, _ = _run_batch(batch)
    ref_lab, ref_it = oracle_batch(batch)
    assert np.array_equal(lab, ref_lab)
    assert np.array_equal(iters, ref_it)
    assert st["iterations"] == ref_it.max() and st["converged"]


def test_batch_mixed_shapes_and_empty_graphs():
    rng = np.random.default_rng(12)
    graphs = [oracle.csr_from_edges(0, []), graphgen.rmat(12, 16, seed=21, permute=True),
              oracle.csr_from_edges(1, []), graphgen.grid(60, 0.55, 40, seed=3), oracle.csr_from_edges(0, []),
              oracle.csr_from_edges(3000, [(0, i) for i in range(1, 3000)])]
    for _ in range(40):
        n = int(rng.integers(1, 3000))
        m = int(rng.integers(0, 4 * n))
        e = {(int(a), int(b)) for a, b in zip(rng.integers(n, size=m), rng.integers(n, size=m)) if a != b}
        graphs.append(oracle.csr_from_edges(n, sorted({(min(a, b), max(a, b)) for a, b in e})))
    batch = graphgen.Batch.from_graphs(graphs)
    for items in (4, 8, 16):
        lab, iters, st, _ = _run_batch(batch, k2_items=items)
        ref_lab, ref_it = oracle_batch(batch)
        assert np.array_equal(lab, ref_lab)
        assert np.array_equal(iters, ref_it)
        assert iters[0] == 0 and iters[4] == 0 and iters[2] == 1


def test_batch_equals_per_graph_calls():
    import paper_1910_05971_gb300 as fsv
    batch = graphgen.er_batch(48, seed=77, nmax=20000)
    lab, iters, _, _ = _run_batch(batch)
    with fsv.FastSV(rowptr_bits=32) as s:
        for g in range(batch.num_graphs):
            rp, ci = batch.graph(g)
            one = s.cc(to_dev(rp, np.int32), to_dev(ci)).cpu().numpy()
            v0, v1 = batch.vtx_off[g], batch.vtx_off[g + 1]
            assert np.array_equal(one, lab[v0:v1])
            assert s.stats()["iterations"] == iters[g]


def test_batch_host_loop_mode():
    batch = graphgen.er_batch(32, seed=5, nmax=5000)
    a = _run_batch(batch)
    b = _run_batch(batch, use_graph=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_batched_config_full():
    """4096 Erdos-Renyi graphs, n log-uniform in [100, 200000], entries per
    vertex uniform in [1.5, 20], seed 4: labels and per-graph iteration
    counts equal the oracle's for every graph."""
    batch = graphgen.er_batch(4096, seed=4)
    lab, iters, st, launches = _run_batch(batch)
    ref_lab, ref_it = oracle_batch(batch)
    assert np.array_equal(lab, ref_lab)
    assert np.array_equal(iters, ref_it)
    assert launches == 5 + 5 * int(ref_it.max())


@pytest.mark.parametrize("sparse_div", [0, 1, 2, 1 << 20])
def test_batch_per_graph_sparse_iterations_are_exact(sparse_div):
    """Each graph of a batch decides after every iteration whether it pushes
    from its changed vertices or runs a full SpMV (Section 4.2); pushing is
    exact, so labels and iteration counts match the oracle whatever the
    threshold (push when the changed vertices' degree sum is at most
    m / sparse_div: 0 never pushes, 1 pushes after every first iteration,
    2^20 practically never)."""
    graphs = [graphgen.rmat(12, 16, seed=31, permute=True), graphgen.grid(60, 0.55, 40, seed=5),
              oracle.csr_from_edges(2000, [(i, i + 1) for i in range(1999)]),
              oracle.csr_from_edges(0, []), oracle.csr_from_edges(1, [])]
    graphs += [graphgen.rmat(9, 8, seed=40 + k) for k in range(20)]
    batch = graphgen.Batch.from_graphs(graphs)
    lab, iters, st, _ = _run_batch(batch, batch_sparse_div=sparse_div)
    ref_lab, ref_it = oracle_batch(batch)
    assert np.array_equal(lab, ref_lab)
    assert np.array_equal(iters, ref_it)
    if sparse_div == 1:
        assert st["sparse_iters"] > 0  # graph 0 pushed in at least one iteration
    if sparse_div == 0:
        assert st["sparse_iters"] == 0

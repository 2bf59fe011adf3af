"""GPU parity of the convergence ablation sv1..sv4 and of the asynchronous mode.

The ablation variants (Section 5.2: Algorithm 1, then the optimizations of
Sections 3.1-3.4 one at a time) are deterministic per iteration, so the
device pointer graph after every iteration, the iteration count and the
per-iteration count of changed entries of f must equal the oracle's exactly.
The asynchronous mode (one parent vector read and written in place, the
concurrent form Section 2.4 mentions) has schedule-dependent intermediate
states: its labels must equal the component minima exactly, and a capped run
must leave a valid pointer graph (every f[u] <= u, inside u's component).
"""
import itertools
import json
import os

import numpy as np
import pytest

import graphgen
import oracle
from gpu_util import Solver, gpu_solve, per_iteration_parity, ragged_graphs, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sv_ablation_hand_traces.json")


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_hand_traces(case, variant):
    import paper_1910_05971_gb300 as fsv
    exp = case["variants"].get(f"sv{variant}")
    if exp is None:
        pytest.skip("no hand trace for this variant")
    rp, ci = oracle.csr_from_edges(case["n"], case["edges"])
    lab, st = gpu_solve(rp, ci, variant=variant)
    assert lab.tolist() == case["labels"]
    assert st["iterations"] == exp["iterations"]
    assert st["changed_per_iter"] == exp["changed"]
    for k, f_exp in enumerate(exp["f_after"], start=1):
        got, stk = gpu_solve(rp, ci, variant=variant, max_iters=k)
        assert got.tolist() == f_exp, f"after iteration {k}"
        assert stk["status"] == (fsv.FASTSV_OK if exp["changed"][k - 1] == 0 else fsv.FASTSV_ERR_MAX_ITERS)


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_exhaustive_small_graphs(variant):
    s = Solver(variant=variant)
    try:
        for n in range(1, 6):
            pairs = list(itertools.combinations(range(n), 2))
            for mask in range(1 << len(pairs)):
                edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
                rp, ci = oracle.csr_from_edges(n, edges)
                f, it, _, ch = oracle.fastsv(rp, ci, form=f"sv{variant}")
                got, st = s.solve(rp, ci)
                assert np.array_equal(got, f), (n, edges)
                assert st["iterations"] == it and st["changed_per_iter"] == ch.tolist()
    finally:
        s.close()


@pytest.mark.parametrize("bits", [32, 64])
@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_per_iteration_parity_ragged(variant, bits):
    for rp, ci in ragged_graphs():
        per_iteration_parity(rp, ci, bits=bits, variant=variant, max_check=24)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5])
def test_larger_graphs_match_oracle(variant):
    """R-MAT scale 16 and a near-percolation lattice: labels, iteration count
    and the whole changed-entry trace."""
    graphs = [graphgen.rmat(16, 16, seed=1, permute=True), graphgen.grid(300, 0.55, 2000, seed=3)]
    for rp, ci in graphs:
        f, it, conv, ch = oracle.fastsv(rp, ci, form=f"sv{variant}")
        got, st = gpu_solve(rp, ci, variant=variant)
        assert conv and np.array_equal(got, f)
        assert st["iterations"] == it and st["converged"]
        assert st["changed_per_iter"] == ch[:64].tolist()


def test_variant5_is_the_default_iteration():
    rp, ci = graphgen.rmat(14, 8, seed=4, permute=True)
    a, sa = gpu_solve(rp, ci)
    b, sb = gpu_solve(rp, ci, variant=5)
    assert np.array_equal(a, b) and sa["iterations"] == sb["iterations"]
    assert sa["changed_per_iter"] == sb["changed_per_iter"]


# ---------------------------------------------------------------------------
# asynchronous mode
# ---------------------------------------------------------------------------

def _async_graphs():
    out = ragged_graphs()
    out.append(graphgen.rmat(16, 16, seed=1, permute=True))
    out.append(graphgen.grid(300, 0.55, 2000, seed=3))
    out.append(graphgen.grid(200, 0.45, 0, seed=8))      # below percolation: many components
    out.append(oracle.csr_from_edges(6, []))               # no edges at all
    n = 5000                                               # one long path, ids shuffled
    perm = np.random.default_rng(6).permutation(n)
    out.append(oracle.csr_from_edges(n, [(int(perm[i]), int(perm[i + 1])) for i in range(n - 1)]))
    return out


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("bits", [32, 64])
def test_async_labels_are_component_minima(bits, use_graph):
    import paper_1910_05971_gb300 as fsv
    s = Solver(bits=bits, mode=fsv.FASTSV_MODE_ASYNC, use_graph=use_graph)
    try:
        for rp, ci in _async_graphs():
            got, st = s.solve(rp, ci)
            assert st["status"] == fsv.FASTSV_OK and st["converged"]
            assert np.array_equal(got, oracle.uf(rp, ci))
            assert st["iterations"] >= 1
            tr = st["changed_per_iter"]
            assert tr[-1] == 0 and all(c > 0 for c in tr[:-1])  # stops at the first quiet iteration
    finally:
        s.close()


def test_async_capped_run_leaves_a_valid_pointer_graph():
    import paper_1910_05971_gb300 as fsv
    rp, ci = graphgen.grid(300, 0.55, 2000, seed=3)
    ref = oracle.uf(rp, ci)
    n = len(rp) - 1
    for k in (1, 2):
        got, st = gpu_solve(rp, ci, mode=fsv.FASTSV_MODE_ASYNC, max_iters=k)
        assert st["status"] == fsv.FASTSV_ERR_MAX_ITERS and st["iterations"] == k
        assert (got <= np.arange(n)).all() and (got >= 0).all()
        assert np.array_equal(ref[got], ref)  # every parent lies in the vertex's component


def test_async_and_ablation_are_single_graph_only():
    import paper_1910_05971_gb300 as fsv
    torch = pytest.importorskip("torch")
    batch = graphgen.er_batch(4, seed=3, nmin=50, nmax=200)
    for kw in ({"mode": fsv.FASTSV_MODE_ASYNC}, {"variant": 2}):
        with fsv.FastSV(rowptr_bits=32, **kw) as s:
            with pytest.raises(fsv.FastSVError) as ei:
                s.cc_batched(to_dev(batch.vtx_off), to_dev(batch.edge_off), to_dev(batch.row_ptr, np.int32),
                             to_dev(batch.col_idx, np.int32))
            assert ei.value.status == fsv.FASTSV_ERR_UNSUPPORTED
            st = fsv._lib.fastsv_pool_create(s.h, 1 << 20, 4)
            assert st == fsv.FASTSV_ERR_UNSUPPORTED
    del torch

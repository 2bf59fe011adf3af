"""The allocation-free entry point fastsv_cc_noalloc, called through the C ABI.

It serves callers that must not allocate device memory while they run (a
framework that has reserved all device memory in its own pool, latency-
critical loops where cudaMalloc/cudaFree would synchronise the device).  It
runs its own kernels (one warp per row), so its labels and iteration counts
are checked against the CPU oracle (integer results: exact), and against the
regular entry point fastsv_cc on two calls in a row -- the second call finds
the first call's leftovers in the shared built-in scratch array.  Edge cases:
a hub row of more than 10^5 entries, exactly FASTSV_NOALLOC_MAX_VERTICES
vertices, the iteration cap, no vertices, and vertices without any entry
(col_idx may then be NULL).
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def _regular(rp, ci):
    """Labels and iterations from the regular (allocating) entry point."""
    import paper_1910_05971_gb300 as fsv
    import torch
    with fsv.FastSV(rowptr_bits=32) as s:
        lab = s.cc(torch.from_numpy(rp.astype(np.int32)).cuda(), torch.from_numpy(ci).cuda())
        return lab.cpu().numpy(), s.stats()["iterations"]


def _noalloc(rp, ci, max_iters=4096):
    import paper_1910_05971_gb300 as fsv
    import torch
    n = len(rp) - 1
    rp_d = torch.from_numpy(rp.astype(np.int32)).cuda()
    ci_d = torch.from_numpy(ci).cuda() if len(ci) else None
    lab = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    st, it = fsv.fastsv_cc_noalloc(n, rp_d.data_ptr(), ci_d.data_ptr() if ci_d is not None else None,
                                   lab.data_ptr(), max_iters, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    return st, lab.cpu().numpy()[:n], it, free_before - free_after


def _oracle(rp, ci, max_iters=0):
    f, it, conv, _ = oracle.fastsv(rp, ci, max_iters=max_iters, form="omp")
    return f, it, conv


def _hub_graph():
    """A star of 150,001 vertices (row 0 holds 150,000 entries) joined to a
    sparse tail of paths and isolated vertices."""
    n = 200_000
    edges = [(0, i) for i in range(1, 150_001)]
    edges += [(i, i + 1) for i in range(150_001, 199_000) if i % 97]
    return oracle.csr_from_edges(n, edges)


def test_noalloc_matches_oracle_and_regular_entry_point_twice():
    import paper_1910_05971_gb300 as fsv
    graphs = [graphgen.rmat(16, 16, seed=1, permute=True), graphgen.grid(600, 0.55, 5000, seed=3)]
    assert all(len(rp) - 1 <= fsv.FASTSV_NOALLOC_MAX_VERTICES for rp, _ in graphs)
    for call, (rp, ci) in enumerate(graphs):
        st, lab, it, grown = _noalloc(rp, ci)
        f, it_ref, conv = _oracle(rp, ci)
        assert conv and st == fsv.FASTSV_OK
        assert np.array_equal(lab, f)
        assert it == it_ref
        reg_lab, reg_it = _regular(rp, ci)
        assert np.array_equal(lab, reg_lab) and it == reg_it
        if call == 1:
            # the second call finds its scratch set up: no device memory taken
            assert grown == 0


def test_noalloc_hub_row():
    import paper_1910_05971_gb300 as fsv
    rp, ci = _hub_graph()
    assert int(np.diff(rp).max()) > 100_000
    st, lab, it, _ = _noalloc(rp, ci)
    f, it_ref, conv = _oracle(rp, ci)
    assert st == fsv.FASTSV_OK and conv
    assert np.array_equal(lab, f) and it == it_ref
    assert np.array_equal(lab, oracle.uf(rp, ci))


def test_noalloc_at_the_vertex_limit():
    import paper_1910_05971_gb300 as fsv
    side = 1024
    assert side * side == fsv.FASTSV_NOALLOC_MAX_VERTICES
    rp, ci = graphgen.grid(side, 0.55, 0, seed=17)
    st, lab, it, _ = _noalloc(rp, ci)
    f, it_ref, conv = _oracle(rp, ci)
    assert st == fsv.FASTSV_OK and conv
    assert np.array_equal(lab, f) and it == it_ref


def test_noalloc_iteration_cap_returns_partial_state():
    import paper_1910_05971_gb300 as fsv
    rp, ci = graphgen.grid(300, 0.55, 0, seed=5)
    _, it_full, _ = _oracle(rp, ci)
    k = 3
    assert it_full > k
    st, lab, it, _ = _noalloc(rp, ci, max_iters=k)
    f, it_ref, conv = _oracle(rp, ci, max_iters=k)
    assert st == fsv.FASTSV_ERR_MAX_ITERS and it == k == it_ref and not conv
    assert np.array_equal(lab, f)  # Algorithm 2's pointer graph after k iterations


def test_noalloc_empty_and_edgeless():
    import paper_1910_05971_gb300 as fsv
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    st, it = fsv.fastsv_cc_noalloc(0, None, None, None, 4096, stream)
    assert st == fsv.FASTSV_OK and it == 0
    n = 777
    rp = np.zeros(n + 1, dtype=np.int64)
    st, lab, it, _ = _noalloc(rp, np.zeros(0, np.int32))  # col_idx NULL: no entries
    f, it_ref, _ = _oracle(rp, np.zeros(0, np.int32))
    assert st == fsv.FASTSV_OK and np.array_equal(lab, np.arange(n)) and np.array_equal(lab, f)
    assert it == it_ref == 1


def test_noalloc_rejects_too_many_vertices():
    import paper_1910_05971_gb300 as fsv
    import torch
    n = fsv.FASTSV_NOALLOC_MAX_VERTICES + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    lab = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    st, it = fsv.fastsv_cc_noalloc(n, rp.data_ptr(), None, lab.data_ptr(), 4096,
                                   torch.cuda.current_stream().cuda_stream)
    assert st == fsv.FASTSV_ERR_UNSUPPORTED and it == 0
    assert int(lab.min().item()) == 7 and int(lab.max().item()) == 7

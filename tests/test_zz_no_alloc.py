"""The allocation-free entry point fastsv_cc_noalloc, called through the C ABI.

It serves callers that must not allocate device memory while they run (a
framework that has reserved all device memory in its own pool, latency-
critical loops where cudaMalloc/cudaFree would synchronise the device).  Its
labels and iteration counts must equal those of the regular entry point
fastsv_cc (integer results: exact), on two calls in a row -- the second call
finds the first call's leftovers in the shared built-in scratch array.
"""
import numpy as np
import pytest

import graphgen

pytestmark = pytest.mark.gpu


def _regular(rp, ci):
    """Labels and iterations from the regular (allocating) entry point."""
    import paper_1910_05971_gb300 as fsv
    import torch
    with fsv.FastSV(rowptr_bits=32) as s:
        lab = s.cc(torch.from_numpy(rp.astype(np.int32)).cuda(), torch.from_numpy(ci).cuda())
        return lab.cpu().numpy(), s.stats()["iterations"]


def _noalloc(rp, ci):
    import paper_1910_05971_gb300 as fsv
    import torch
    rp_d = torch.from_numpy(rp.astype(np.int32)).cuda()
    ci_d = torch.from_numpy(ci).cuda()
    lab = torch.full((len(rp) - 1,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    st, it = fsv.fastsv_cc_noalloc(len(rp) - 1, rp_d.data_ptr(), ci_d.data_ptr(), lab.data_ptr(), 4096,
                                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    return st, lab.cpu().numpy(), it, free_before - free_after


def test_noalloc_matches_regular_entry_point_twice():
    import paper_1910_05971_gb300 as fsv
    graphs = [graphgen.rmat(16, 16, seed=1, permute=True), graphgen.grid(600, 0.55, 5000, seed=3)]
    assert all(len(rp) - 1 <= fsv.FASTSV_NOALLOC_MAX_VERTICES for rp, _ in graphs)
    for call, (rp, ci) in enumerate(graphs):
        st, lab, it, grown = _noalloc(rp, ci)
        ref_lab, ref_it = _regular(rp, ci)
        assert st == fsv.FASTSV_OK
        assert np.array_equal(lab, ref_lab)
        assert it == ref_it
        if call == 1:
            # the second call finds its scratch set up: no device memory taken
            assert grown == 0


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

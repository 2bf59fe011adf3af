"""GPU parity tests: the CUDA path (through the C ABI) against the CPU oracle.

Labels and iteration counts must match exactly (integer work: bit-exact);
in sync mode the pointer graph after every iteration must match too.
"""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle
from gpu_util import Solver, gpu_solve, oracle_batch, per_iteration_parity, ragged_graphs, to_dev, workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "alg2_hand_traces.json")


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_traces(case):
    import paper_1910_05971_gb300 as fsv
    rp, ci = oracle.csr_from_edges(case["n"], case["edges"])
    lab, st = gpu_solve(rp, ci)
    assert lab.tolist() == case["labels"]
    assert st["iterations"] == case["iterations"]
    assert st["changed_per_iter"] == case["changed"]
    for k, f_exp in enumerate(case["f_after"], start=1):
        got, stk = gpu_solve(rp, ci, max_iters=k)
        assert got.tolist() == f_exp, f"after iteration {k}"
        expect = fsv.FASTSV_OK if case["changed"][k - 1] == 0 else fsv.FASTSV_ERR_MAX_ITERS
        assert stk["status"] == expect


def test_exhaustive_small_graphs():
    import itertools
    s = Solver()
    try:
        for n in range(1, 6):
            pairs = list(itertools.combinations(range(n), 2))
            for mask in range(1 << len(pairs)):
                edges = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
                rp, ci = oracle.csr_from_edges(n, edges)
                f, it, _, ch = oracle.fastsv(rp, ci)
                got, st = s.solve(rp, ci)
                assert np.array_equal(got, f), (n, edges)
                assert st["iterations"] == it and st["changed_per_iter"] == ch.tolist()
    finally:
        s.close()


def _ragged_graphs():
    return ragged_graphs()


@pytest.mark.parametrize("threads", [64, 256])
@pytest.mark.parametrize("items", [4, 8, 16])
@pytest.mark.parametrize("bits", [32, 64])
def test_per_iteration_parity_ragged(items, bits, threads):
    for rp, ci in _ragged_graphs():
        per_iteration_parity(rp, ci, bits=bits, k2_items=items, k2_threads=threads)


@pytest.mark.parametrize("col_blocks", [2, 3, 4, 16])
def test_per_iteration_parity_column_blocks(col_blocks):
    """Column-blocked hooking (one pass per column range, partial minima
    hooked directly) reproduces Algorithm 2 iteration by iteration."""
    for bits in (32, 64):
        for items, threads in ((4, 64), (8, 256), (16, 64)):
            for rp, ci in _ragged_graphs():
                per_iteration_parity(rp, ci, bits=bits, k2_items=items, k2_threads=threads, col_blocks=col_blocks)


def test_column_blocks_with_unsorted_rows():
    """Rows need not be sorted: shuffle every row and compare."""
    rng = np.random.default_rng(4)
    rp, ci = graphgen.rmat(12, 16, seed=9, permute=True)
    ci = ci.copy()
    for u in range(len(rp) - 1):
        seg = ci[rp[u]:rp[u + 1]]
        rng.shuffle(seg)
    f, it, _, ch = oracle.fastsv(rp, ci)
    for nb in (1, 4, 8):
        got, st = gpu_solve(rp, ci, col_blocks=nb)
        assert np.array_equal(got, f) and st["iterations"] == it and st["changed_per_iter"] == ch.tolist()


@pytest.mark.parametrize("k", [2, 3])
def test_column_blocks_with_one_descent_at_a_tile_boundary(k):
    """The only unsorted pair of the graph lies in a hub row and straddles a
    boundary of the 1024-item merge-path tiles along which the block copy is
    cut, with its two ids in different column blocks: the hub's runs of one
    block then come from several tiles and must merge atomically, and the
    solve must still reproduce Algorithm 2."""
    n = 4096
    row0 = [1] + list(range(3001, 4024))      # 1024 entries: the hub's row starts at entry 1024
    hub = [0] + list(range(2, 3001))          # vertex 1
    edges = [(0, v) for v in row0] + [(1, v) for v in hub[1:]] + [(4024 + i, 4025 + i) for i in range(0, 70, 2)]
    rp, ci = oracle.csr_from_edges(n, edges)
    ci = ci.copy()
    assert rp[1] - rp[0] == 1024 and ci[rp[1]:rp[2]].tolist() == hub
    # entry y of row u sits at merge-path diagonal u + y; a tile starts every
    # 1024 diagonals, so hub entry j starts tile k for j = 1024k - 1025
    j = 1024 * k - 1025
    y = int(rp[1]) + j
    assert (1 + y) % 1024 == 0
    ci[y - 1], ci[y] = ci[y], ci[y - 1]
    assert ci[y - 1] // 1024 != ci[y] // 1024      # 4 blocks of 1024 ids
    f, it, _, ch = oracle.fastsv(rp, ci)
    for nb in (1, 4):
        got, st = gpu_solve(rp, ci, col_blocks=nb)
        assert np.array_equal(got, f) and st["iterations"] == it and st["changed_per_iter"] == ch.tolist()


def test_host_loop_mode_matches():
    rp, ci = graphgen.rmat(13, 8, seed=2, permute=True)
    f, it, _, ch = oracle.fastsv(rp, ci)
    got, st = gpu_solve(rp, ci, use_graph=False)
    assert np.array_equal(got, f) and st["iterations"] == it
    assert st["ms_k2"] > 0 and st["ms_k3"] > 0


def test_edge_cases():
    import paper_1910_05971_gb300 as fsv
    torch = pytest.importorskip("torch")
    with fsv.FastSV() as s:
        lab = s.cc(torch.zeros(1, dtype=torch.int64, device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"))
        assert lab.numel() == 0 and s.stats()["iterations"] == 0
    rp, ci = oracle.csr_from_edges(1, [])
    got, st = gpu_solve(rp, ci)
    assert got.tolist() == [0] and st["iterations"] == 1
    rp, ci = oracle.csr_from_edges(500, [])
    got, st = gpu_solve(rp, ci)
    assert got.tolist() == list(range(500)) and st["iterations"] == 1
    # self-loops and duplicate entries change nothing
    rng = np.random.default_rng(5)
    edges = sorted({(int(a), int(b)) for a, b in zip(rng.integers(400, size=300), rng.integers(400, size=300)) if a < b})
    noisy = edges + edges[:50] + [(i, i) for i in range(0, 400, 9)]
    f, it, _, ch = oracle.fastsv(*oracle.csr_from_edges(400, edges))
    for nb in (1, 4):  # also through the column-block copy (rows with repeated ids count as sorted)
        got, st = gpu_solve(*oracle.csr_from_edges(400, noisy), col_blocks=nb)
        assert np.array_equal(got, f) and st["iterations"] == it and st["changed_per_iter"] == ch.tolist()


def test_iteration_cap_reports_partial_state():
    import paper_1910_05971_gb300 as fsv
    n = 4000
    rp, ci = oracle.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    f2, it2, conv, _ = oracle.fastsv(rp, ci, max_iters=2)
    assert not conv
    got, st = gpu_solve(rp, ci, max_iters=2)
    assert st["status"] == fsv.FASTSV_ERR_MAX_ITERS and st["iterations"] == 2
    assert np.array_equal(got, f2)
    with pytest.raises(fsv.FastSVError):
        with fsv.FastSV(max_iters=2) as s:
            s.cc(to_dev(rp), to_dev(ci))


def test_validation_rejects_malformed_csr():
    import paper_1910_05971_gb300 as fsv
    rp, ci = oracle.csr_from_edges(6, [(0, 1), (1, 2), (3, 4)])
    got, st = gpu_solve(rp, ci, validate=2)
    assert st["status"] == fsv.FASTSV_OK
    bad = ci.copy()
    bad[0] = 17
    with fsv.FastSV(validate=1) as s:
        with pytest.raises(fsv.FastSVError) as e:
            s.cc(to_dev(rp), to_dev(bad))
        assert e.value.status == fsv.FASTSV_ERR_INVALID_GRAPH
    badrp = rp.copy()
    badrp[2], badrp[3] = badrp[3], badrp[2]
    with fsv.FastSV(validate=1) as s:
        with pytest.raises(fsv.FastSVError) as e:
            s.cc(to_dev(badrp), to_dev(ci))
        assert e.value.status == fsv.FASTSV_ERR_INVALID_GRAPH
    rp_a, ci_a = oracle.csr_from_edges(4, [(0, 1), (2, 3)])
    ci_a = ci_a.copy()
    ci_a[ci_a.tolist().index(0)] = 2  # row 1 now points to 2, row 2 does not point back
    with fsv.FastSV(validate=2) as s:
        with pytest.raises(fsv.FastSVError) as e:
            s.cc(to_dev(rp_a), to_dev(np.sort(ci_a)))
        assert e.value.status == fsv.FASTSV_ERR_INVALID_GRAPH


def test_malformed_csr_without_validation_stays_in_bounds():
    """With validation off a malformed CSR is outside the contract, but the
    kernels clamp every index, so the call completes and the handle stays usable."""
    import paper_1910_05971_gb300 as fsv
    rp, ci = oracle.csr_from_edges(6, [(0, 1), (1, 2), (3, 4)])
    bad = ci.copy()
    bad[0] = 1 << 30
    with fsv.FastSV() as s:
        s.cc(to_dev(rp), to_dev(bad), check_status=False)
        s.stats()
        lab = s.cc(to_dev(rp), to_dev(ci))
        assert lab.cpu().tolist() == [0, 0, 0, 3, 3, 5]


def test_allocation_failure_is_reported_and_recoverable():
    import paper_1910_05971_gb300 as fsv
    rp, ci = graphgen.rmat(10, 8, seed=4)
    f, it, _, _ = oracle.fastsv(rp, ci)
    with fsv.FastSV(fail_alloc_after=1) as s:
        with pytest.raises(fsv.FastSVError) as e:
            s.cc(to_dev(rp), to_dev(ci))
        assert e.value.status == fsv.FASTSV_ERR_OOM
        lab = s.cc(to_dev(rp), to_dev(ci))
        assert np.array_equal(lab.cpu().numpy(), f)


def test_host_buffer_entry_point():
    import paper_1910_05971_gb300 as fsv
    torch = pytest.importorskip("torch")
    rp, ci = graphgen.rmat(14, 16, seed=8, permute=True)
    f, it, _, _ = oracle.fastsv(rp, ci, form="omp")
    rp_h = torch.from_numpy(rp).pin_memory()
    ci_h = torch.from_numpy(ci).pin_memory()
    with fsv.FastSV() as s:
        lab = s.cc_host(rp_h, ci_h)
        assert np.array_equal(lab.numpy(), f)
        assert s.stats()["iterations"] == it


@pytest.mark.parametrize("col_blocks", [2, 4, 16])
def test_host_buffer_entry_point_column_blocked(col_blocks):
    """fastsv_cc_host on a column-blocked solve copies col_idx in chunks that
    overlap the first iteration (each chunk's tiles run once their entries
    have landed; from the second call on, each chunk is also split into the
    column blocks right away): labels, iterations and the per-iteration trace
    must still be Algorithm 2's, on repeated calls into the same device
    buffers."""
    import paper_1910_05971_gb300 as fsv
    torch = pytest.importorskip("torch")
    for seed in (8, 9):
        rp, ci = graphgen.rmat(13, 16, seed=seed, permute=True)
        f, it, _, ch = oracle.fastsv(rp, ci, form="omp")
        rp_h = torch.from_numpy(rp).pin_memory()
        ci_h = torch.from_numpy(ci).pin_memory()
        with fsv.FastSV(col_blocks=col_blocks) as s:
            for _ in range(2):
                lab = s.cc_host(rp_h, ci_h)
                st = s.stats()
                assert st["col_blocks"] > 1
                assert np.array_equal(lab.numpy(), f) and st["iterations"] == it
                assert st["changed_per_iter"] == ch.tolist()


def test_host_buffer_column_blocked_runs_outgrow_an_earlier_call():
    """The chunk-by-chunk block copy of fastsv_cc_host sizes its run arrays
    from the handle's earlier calls; a larger graph after a smaller one
    overflows them, and the call must notice, grow them and copy again."""
    import paper_1910_05971_gb300 as fsv
    torch = pytest.importorskip("torch")
    small = graphgen.rmat(11, 16, seed=3, permute=True)
    large = graphgen.rmat(13, 16, seed=4, permute=True)
    with fsv.FastSV(col_blocks=4) as s:
        for rp, ci in (small, large, large, small):
            f, it, _, ch = oracle.fastsv(rp, ci, form="omp")
            lab = s.cc_host(torch.from_numpy(rp).pin_memory(), torch.from_numpy(ci).pin_memory())
            st = s.stats()
            assert st["col_blocks"] == 4
            assert np.array_equal(lab.numpy(), f) and st["iterations"] == it
            assert st["changed_per_iter"] == ch.tolist()


def test_non_default_stream_and_launch_count():
    import paper_1910_05971_gb300 as fsv
    torch = pytest.importorskip("torch")
    rp, ci = graphgen.rmat(12, 8, seed=6, permute=True)
    f, it, _, _ = oracle.fastsv(rp, ci)
    stream = torch.cuda.Stream()
    with fsv.FastSV() as s:
        with torch.cuda.stream(stream):
            rp_d, ci_d = to_dev(rp), to_dev(ci)
            lab = s.cc(rp_d, ci_d, stream=stream)
        stream.synchronize()
        assert np.array_equal(lab.cpu().numpy(), f)
        # set-up (3) + finish (1) + five kernels per device-loop iteration
        assert s.kernel_launches() == 4 + 5 * it


@pytest.mark.parametrize("col_blocks", [1, 2])
def test_launch_count_over_unsynchronised_calls(col_blocks):
    """Calls issued back to back without a status check in between are all
    counted: the device loop keeps a running total of its launches."""
    import paper_1910_05971_gb300 as fsv
    rp, ci = graphgen.rmat(12, 16, seed=6, permute=True)
    _, it, _, _ = oracle.fastsv(rp, ci)
    rp_d, ci_d = to_dev(rp), to_dev(ci)
    with fsv.FastSV(col_blocks=col_blocks) as s:
        lab = s.cc(rp_d, ci_d)
        one = s.kernel_launches()
        if col_blocks == 1:
            assert one == 4 + 5 * it
        else:
            # set-up (3), the first iteration on the original CSR (4), the
            # scan of its block counts and the blocks' layout (4), the check
            # of the copy's totals (1), the block split and the blocks'
            # set-up (4), finish (1); then 4 + col_blocks kernels per
            # device-loop iteration
            assert one == 17 + (4 + col_blocks) * (it - 1)
        for _ in range(5):
            s.cc(rp_d, ci_d, lab, check_status=False)
        s.check_last()
        assert s.kernel_launches() == 6 * one


# ---------------------------------------------------------------------------
# the named workloads at full size
# ---------------------------------------------------------------------------

def test_rmat_s16_full_per_iteration():
    rp, ci = workload("rmat_s16")
    k = per_iteration_parity(rp, ci, bits=32)
    f, it, _, _ = oracle.fastsv(rp, ci)
    assert k == it
    assert np.array_equal(f, oracle.uf(rp, ci))


def test_grid_full():
    rp, ci = workload("grid_4096_p055_iso1M")
    ref = oracle.uf(rp, ci)
    f, it, conv, ch = oracle.fastsv(rp, ci, form="omp")
    assert conv and np.array_equal(f, ref)
    got, st = gpu_solve(rp, ci, bits=32)
    assert np.array_equal(got, ref)
    assert st["iterations"] == it
    assert st["changed_per_iter"] == ch.tolist()[:64]


@pytest.mark.slow
def test_rmat_s26_full():
    rp, ci = workload("rmat_s26_perm")
    got, st = gpu_solve(rp, ci, bits=64)
    ref = oracle.uf(rp, ci)
    assert np.array_equal(got, ref)
    f, it, conv, ch = oracle.fastsv(rp, ci, form="omp")
    assert conv and np.array_equal(f, ref)
    assert st["iterations"] == it
    assert st["changed_per_iter"] == ch.tolist()[:64]


# ---------------------------------------------------------------------------
# sparse iterations (push from the vertices whose grandparent changed)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("sparse_div", [0, 1, 4, 1 << 20])
def test_per_iteration_parity_sparse_modes(sparse_div):
    """Iterations that push from the changed vertices instead of a full SpMV
    (sparse_div = 1: every iteration after the first) still reproduce
    Algorithm 2's pointer graph after every iteration."""
    for rp, ci in _ragged_graphs():
        per_iteration_parity(rp, ci, sparse_div=sparse_div)
    for rp, ci in _ragged_graphs()[-3:]:
        per_iteration_parity(rp, ci, sparse_div=sparse_div, col_blocks=4, bits=32)


def test_sparse_iterations_are_used_and_exact():
    # R-MAT: late frontiers are small, so the default threshold pushes
    rp, ci = graphgen.rmat_s16()
    f, it, _, ch = oracle.fastsv(rp, ci)
    dense, st_d = gpu_solve(rp, ci, sparse_div=0, bits=32)
    sparse, st_s = gpu_solve(rp, ci, bits=32)
    assert st_d["sparse_iters"] == 0 and st_s["sparse_iters"] > 0
    # lattice: frontiers stay large; forcing a push in every iteration after
    # the first must still be exact
    rpg, cig = graphgen.grid(300, 0.55, 100, seed=7)
    fg, itg, _, chg = oracle.fastsv(rpg, cig)
    always, st_a = gpu_solve(rpg, cig, sparse_div=1)
    assert st_a["sparse_iters"] == itg - 1
    for got, st, ref, n_it, trace in ((dense, st_d, f, it, ch), (sparse, st_s, f, it, ch), (always, st_a, fg, itg, chg)):
        assert np.array_equal(got, ref) and st["iterations"] == n_it and st["changed_per_iter"] == trace.tolist()


def test_tuning_cache_entry_is_applied(tmp_path):
    """A tuning-cache entry for the call's shape class replaces the kernel
    choices (here: column blocks and tile shape forced, pushes off); the
    result stays Algorithm 2's, iteration by iteration."""
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300 import tune
    rp, ci = graphgen.rmat(12, 16, seed=6, permute=True)
    f, it, _, ch = oracle.fastsv(rp, ci)
    key = fsv.fastsv_tune_key(fsv.TUNE_SINGLE, len(rp) - 1, len(ci), 1, 64)
    path = str(tmp_path / "cache.txt")
    tune.write_cache(path, {key: dict(k2_items=16, k2_threads=64, col_blocks=4, sparse_div=0, batch_sparse_div=0)})
    with fsv.FastSV(tune_cache=path) as s:
        lab = s.cc(to_dev(rp), to_dev(ci))
        st = s.stats()
    assert st["tuned"] and st["col_blocks"] == 4 and st["sparse_iters"] == 0 and st["block_runs"] > 0
    assert np.array_equal(lab.cpu().numpy(), f) and st["iterations"] == it
    assert st["changed_per_iter"] == ch.tolist()
    rp2, ci2 = graphgen.rmat(10, 8, seed=1)  # another shape class: the handle's own options
    with fsv.FastSV(tune_cache=path) as s:
        lab2 = s.cc(to_dev(rp2), to_dev(ci2))
        st2 = s.stats()
    assert not st2["tuned"] and st2["col_blocks"] == 1
    assert np.array_equal(lab2.cpu().numpy(), oracle.uf(rp2, ci2))
    with pytest.raises(fsv.FastSVError):
        fsv.FastSV(tune_cache=str(tmp_path / "missing.txt"))

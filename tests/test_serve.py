"""GPU tests of the serving pool: a graph's labels and iteration count are the
same alone and inside a continuously changing batch (tolerance 0)."""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def _graphs(count, seed=1):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        k = int(rng.integers(4))
        if k == 0:
            out.append(graphgen.rmat(int(rng.integers(6, 13)), int(rng.integers(8, 33)), seed=100 + i))
        elif k == 1:
            out.append(graphgen.grid(int(rng.integers(5, 80)), float(rng.uniform(0.4, 0.9)), 0, seed=200 + i))
        elif k == 2:
            out.append(oracle.csr_from_edges(int(rng.integers(1, 40)), []))
        else:
            n = int(rng.integers(2, 3000))
            out.append(oracle.csr_from_edges(n, [(j, j + 1) for j in range(n - 1)]))
    return [(rp.astype(np.int32), ci.astype(np.int32)) for rp, ci in out]


def _alone(graphs):
    res = []
    for rp, ci in graphs:
        f, it, conv, _ = oracle.fastsv(rp, ci)
        assert conv
        res.append((f, it))
    return res


def test_pool_continuous_admission_matches_alone():
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300.serve import PoolBackend
    graphs = _graphs(40)
    ref = _alone(graphs)
    pool = PoolBackend(64 << 20, 16)
    labels = [np.empty(max(len(rp) - 1, 1), np.int32) for rp, _ in graphs]
    pending = list(range(len(graphs)))
    slot_of = {}
    done = {}
    steps = 0
    while len(done) < len(graphs):
        # admit at most 3 per step so admissions interleave with running graphs
        for _ in range(3):
            if not pending:
                break
            g = pending[0]
            slot = pool.add(graphs[g][0], graphs[g][1], labels[g])
            if slot is None:
                break
            pending.pop(0)
            slot_of[slot] = g
        pool.step(1)
        steps += 1
        fin, _ = pool.poll()
        for slot, iters in fin:
            g = slot_of.pop(slot)
            done[g] = iters
        assert steps < 10000
    for g, (f, it) in enumerate(ref):
        n = len(graphs[g][0]) - 1
        assert np.array_equal(labels[g][:n], f), g
        assert done[g] == it, (g, done[g], it)
    st, used, b = fsv.fastsv_pool_usage(pool.h)
    assert used == 0 and b == 0
    pool.close()


def test_pool_budget_and_full():
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300.serve import PoolBackend
    rp, ci = graphgen.rmat(12, 16, seed=3)
    rp, ci = rp.astype(np.int32), ci.astype(np.int32)
    need = fsv.fastsv_pool_bytes(len(rp) - 1, len(ci))
    pool = PoolBackend(int(need * 2.5), 8)
    labs = [np.empty(len(rp) - 1, np.int32) for _ in range(3)]
    assert pool.add(rp, ci, labs[0]) is not None
    assert pool.add(rp, ci, labs[1]) is not None
    assert pool.add(rp, ci, labs[2]) is None           # budget exhausted: FULL
    big_rp, big_ci = graphgen.rmat(14, 16, seed=3)
    st, _ = fsv.fastsv_pool_add(pool.h, len(big_rp) - 1, big_rp.astype(np.int32).ctypes.data,
                                big_ci.ctypes.data, labs[2].ctypes.data)
    assert st in (fsv.FASTSV_ERR_FULL, fsv.FASTSV_ERR_INVALID_ARG)
    f, it, _, _ = oracle.fastsv(rp, ci)
    finished = []
    for _ in range(100):
        pool.step(2)
        done, active = pool.poll()
        finished += done
        if len(finished) == 2:
            break
    assert len(finished) == 2 and all(i == it for _, i in finished)
    assert np.array_equal(labs[0], f) and np.array_equal(labs[1], f)
    assert pool.add(rp, ci, labs[2]) is not None       # space was returned
    pool.close()


def test_server_mix_equals_alone():
    from paper_1910_05971_gb300.serve import Server
    graphs = _graphs(60, seed=9)
    ref = _alone(graphs)
    with Server(hbm_budget_bytes=32 << 20, max_slots=12, iters_per_step=1) as srv:
        futs = [srv.submit(rp, ci) for rp, ci in graphs]
        res = [f.result(timeout=120) for f in futs]
        summ = srv.summary()
    for (lab, it), (f, it_ref) in zip(res, ref):
        assert np.array_equal(lab, f) and it == it_ref
    assert summ["completed"] == len(graphs) and summ["p99_s"] >= summ["p50_s"]


def test_server_rejects_oversized_request():
    from paper_1910_05971_gb300.serve import Server
    rp, ci = graphgen.rmat(14, 16, seed=1)
    with Server(hbm_budget_bytes=1 << 20, max_slots=4) as srv:
        fut = srv.submit(rp, ci)
        with pytest.raises(ValueError):
            fut.result(timeout=10)


def _oracle_after(rp, ci, k):
    f = np.arange(len(rp) - 1, dtype=np.int32)
    for _ in range(k):
        oracle.iteration(rp, ci, f)
    return f


def _run_to_end(pool, slot_of, done, limit=10000):
    steps = 0
    while slot_of:
        pool.step(1)
        steps += 1
        fin, _ = pool.poll()
        for slot, iters in fin:
            done[slot_of.pop(slot)] = iters
        assert steps < limit


def test_evict_and_restore_resume_exactly():
    """A graph checkpointed after k iterations holds Algorithm 2's f and
    f[f] after k iterations; restored later (into the same pool while others
    run, or into another pool) it finishes with the labels and iteration count
    of an uninterrupted solve."""
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300.serve import PoolBackend
    graphs = [graphgen.grid(80, 0.55, 0, seed=11), graphgen.grid(60, 0.6, 7, seed=12),
              graphgen.rmat(12, 4, seed=13), oracle.csr_from_edges(3000, [(j, j + 1) for j in range(2999)])]
    graphs = [(rp.astype(np.int32), ci.astype(np.int32)) for rp, ci in graphs]
    ref = _alone(graphs)
    assert all(it > 3 for _, it in ref)  # all still iterating after two steps
    # every graph added before a step takes part in it (the checkpoints are
    # compared after exactly two iterations)
    pool = PoolBackend(64 << 20, 8, pool_wait_copies=True)
    other = PoolBackend(64 << 20, 8, pool_wait_copies=True)
    labels = [np.full(len(rp) - 1, -1, np.int32) for rp, _ in graphs]
    slot_of = {}
    for g, (rp, ci) in enumerate(graphs):
        slot_of[pool.add(rp, ci, labels[g])] = g
    pool.step(1)
    pool.step(1)
    assert pool.poll()[0] == []
    _, _, bytes_before = fsv.fastsv_pool_usage(pool.h)
    evicted = {}
    for slot, g in list(slot_of.items()):
        if g in (0, 3):
            ck = pool.evict(slot)
            del slot_of[slot]
            evicted[g] = ck
            rp, ci = graphs[g]
            n = len(rp) - 1
            f = ck[64:64 + 4 * n].view(np.int32)
            gf = ck[64 + 4 * n:64 + 8 * n].view(np.int32)
            assert np.array_equal(f, _oracle_after(rp, ci, 2))
            assert np.array_equal(gf, f[f])
    _, used, bytes_after = fsv.fastsv_pool_usage(pool.h)
    assert used == 2
    assert bytes_before - bytes_after == sum(fsv.fastsv_pool_bytes(len(graphs[g][0]) - 1, len(graphs[g][1]))
                                             for g in evicted)
    pool.step(1)  # the others go on without them
    # graph 0 comes back into the same pool, graph 3 into another one
    rp, ci = graphs[0]
    slot_of[pool.restore(rp, ci, labels[0], evicted[0])] = 0
    other_slots = {}
    rp, ci = graphs[3]
    other_slots[other.restore(rp, ci, labels[3], evicted[3])] = 3
    done = {}
    _run_to_end(pool, slot_of, done)
    _run_to_end(other, other_slots, done)
    for g, (f, it) in enumerate(ref):
        assert np.array_equal(labels[g], f), g
        assert done[g] == it, (g, done[g], it)
    pool.close()
    other.close()


def test_evict_and_restore_errors():
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300.serve import PoolBackend
    rp, ci = graphgen.grid(40, 0.6, 0, seed=21)
    rp, ci = rp.astype(np.int32), ci.astype(np.int32)
    small = oracle.csr_from_edges(2, [(0, 1)])
    small = (small[0].astype(np.int32), small[1].astype(np.int32))
    pool = PoolBackend(16 << 20, 4, pool_wait_copies=True)  # graphs added before a step take part in it
    lab = np.empty(len(rp) - 1, np.int32)
    buf = np.zeros(fsv.fastsv_pool_checkpoint_bytes(len(rp) - 1), np.uint8)
    assert fsv.fastsv_pool_evict(pool.h, 0, buf.ctypes.data) == fsv.FASTSV_ERR_INVALID_ARG  # free slot
    s = pool.add(rp, ci, lab)
    # added but not stepped yet: nothing to checkpoint
    assert fsv.fastsv_pool_evict(pool.h, s, buf.ctypes.data) == fsv.FASTSV_ERR_INVALID_ARG
    lab2 = np.empty(2, np.int32)
    s2 = pool.add(small[0], small[1], lab2)
    pool.step(2)  # the 2-vertex graph finishes in 2 iterations; the lattice does not
    assert fsv.fastsv_pool_evict(pool.h, s2, buf.ctypes.data) == fsv.FASTSV_ERR_INVALID_ARG  # finished
    ck = pool.evict(s)
    bad = ck.copy()
    bad[0] ^= 0xFF
    assert fsv.fastsv_pool_restore(pool.h, len(rp) - 1, rp.ctypes.data, ci.ctypes.data, lab.ctypes.data,
                                   bad.ctypes.data)[0] == fsv.FASTSV_ERR_INVALID_ARG
    # a checkpoint of another graph (n differs)
    assert fsv.fastsv_pool_restore(pool.h, 2, small[0].ctypes.data, small[1].ctypes.data, lab2.ctypes.data,
                                   ck.ctypes.data)[0] == fsv.FASTSV_ERR_INVALID_ARG
    fin, _ = pool.poll()
    assert [x[0] for x in fin] == [s2]
    slot = pool.restore(rp, ci, lab, ck)
    done = {}
    _run_to_end(pool, {slot: 0}, done)
    f, it, _, _ = oracle.fastsv(rp, ci)
    assert np.array_equal(lab, f) and done[0] == it
    pool.close()


@pytest.mark.parametrize("sparse_div", [0, 1])
def test_pool_sparse_iterations_match_alone(sparse_div):
    """Resident graphs choose push or full SpMV per iteration on their own;
    with pushes forced (1) or off (0) every graph still gets its own labels
    and iteration count."""
    from paper_1910_05971_gb300.serve import PoolBackend
    graphs = _graphs(24, seed=7)
    ref = _alone(graphs)
    pool = PoolBackend(64 << 20, 16, batch_sparse_div=sparse_div)
    labels = [np.empty(max(len(rp) - 1, 1), np.int32) for rp, _ in graphs]
    pending = list(range(len(graphs)))
    slot_of, done = {}, {}
    steps = 0
    while len(done) < len(graphs):
        for _ in range(4):
            if not pending:
                break
            slot = pool.add(graphs[pending[0]][0], graphs[pending[0]][1], labels[pending[0]])
            if slot is None:
                break
            slot_of[slot] = pending.pop(0)
        pool.step(1)
        steps += 1
        for slot, iters in pool.poll()[0]:
            done[slot_of.pop(slot)] = iters
        assert steps < 10000
    for g, (f, it) in enumerate(ref):
        n = len(graphs[g][0]) - 1
        assert np.array_equal(labels[g][:n], f), g
        assert done[g] == it, (g, done[g], it)
    pool.close()

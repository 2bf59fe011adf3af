"""Host-side logic of the continuous-batching server, on CPU: a fake pool
backend runs the oracle one Algorithm 2 iteration per step per resident graph.
Checks admission order, back-pressure when the pool is full, rejection of
requests larger than the budget, equality with solving alone, and that a
failing backend fails every outstanding request instead of hanging."""
import threading
import time

import numpy as np
import pytest

import oracle


class FakePool:
    def __init__(self, budget, max_slots, fail_after_steps=None, step_delay=0.0):
        self.budget = budget
        self.max_slots = max_slots
        self.used = 0
        self.slots = {}
        self.admit_order = []
        self.max_resident = 0
        self.steps = 0
        self.fail_after_steps = fail_after_steps
        self.step_delay = step_delay
        self.evicted = 0

    def bytes_for(self, n, m):
        return 4 * (n + 1) + 4 * max(m, 1) + 12 * n

    def add(self, rp, ci, labels):
        b = self.bytes_for(len(rp) - 1, len(ci))
        if len(self.slots) >= self.max_slots or self.used + b > self.budget:
            return None
        slot = next(i for i in range(self.max_slots) if i not in self.slots)
        n = len(rp) - 1
        self.slots[slot] = dict(rp=rp, ci=ci, labels=labels, f=np.arange(n, dtype=np.int32), iters=0,
                                done=n == 0, bytes=b)
        self.used += b
        self.admit_order.append(id(labels))
        self.max_resident = max(self.max_resident, len(self.slots))
        return slot

    def step(self, iters):
        if self.step_delay:
            time.sleep(self.step_delay)
        self.steps += 1
        if self.fail_after_steps is not None and self.steps > self.fail_after_steps:
            raise RuntimeError("device lost (simulated)")
        for s in self.slots.values():
            for _ in range(iters):
                if s["done"]:
                    break
                ch = oracle.iteration(s["rp"], s["ci"], s["f"])
                s["iters"] += 1
                if ch == 0:
                    s["done"] = True

    def evict(self, slot):
        s = self.slots.pop(slot)
        assert not s["done"] and s["iters"] > 0
        self.used -= s["bytes"]
        self.evicted += 1
        return dict(f=s["f"].copy(), iters=s["iters"])

    def restore(self, rp, ci, labels, ck):
        slot = self.add(rp, ci, labels)
        if slot is not None:
            self.slots[slot]["f"] = ck["f"].copy()
            self.slots[slot]["iters"] = ck["iters"]
        return slot

    def poll(self):
        out = []
        for slot in list(self.slots):
            s = self.slots[slot]
            if s["done"]:
                n = len(s["rp"]) - 1
                s["labels"][:n] = s["f"]
                out.append((slot, s["iters"]))
                self.used -= s["bytes"]
                del self.slots[slot]
        return out, len(self.slots)

    def close(self):
        pass


def _graphs(k, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        n = int(rng.integers(1, 300))
        m = int(rng.integers(0, 2 * n))
        e = sorted({(min(a, b), max(a, b)) for a, b in zip(rng.integers(n, size=m), rng.integers(n, size=m)) if a != b})
        out.append(oracle.csr_from_edges(n, e))
    return out


def test_server_matches_alone_with_backpressure():
    from paper_1910_05971_gb300.serve import Server
    graphs = _graphs(50)
    pool = FakePool(budget=20_000, max_slots=4)
    with Server(backend=pool, iters_per_step=1) as srv:
        futs = [srv.submit(rp, ci) for rp, ci in graphs]
        res = [f.result(timeout=60) for f in futs]
        reqs = list(srv.completed)
    for (rp, ci), (lab, it) in zip(graphs, res):
        f, it_ref, _, _ = oracle.fastsv(rp, ci)
        assert np.array_equal(lab, f) and it == it_ref
    assert pool.max_resident <= 4
    # admission follows arrival order (FIFO, no overtaking while full)
    by_labels = {id(r.labels): i for i, r in enumerate(sorted(reqs, key=lambda r: r.t_submit))}
    assert [by_labels[x] for x in pool.admit_order] == sorted(by_labels[x] for x in pool.admit_order)


def test_server_rejects_request_that_never_fits():
    from paper_1910_05971_gb300.serve import Server
    pool = FakePool(budget=500, max_slots=4)
    rp, ci = oracle.csr_from_edges(200, [(i, i + 1) for i in range(199)])
    with Server(backend=pool) as srv:
        with pytest.raises(ValueError):
            srv.submit(rp, ci).result(timeout=10)
        small = oracle.csr_from_edges(3, [(0, 1)])
        lab, it = srv.submit(*small).result(timeout=10)
        assert lab.tolist() == [0, 0, 2] and it == 2


def test_backend_failure_fails_outstanding_requests():
    from paper_1910_05971_gb300.serve import Server
    pool = FakePool(budget=10**9, max_slots=8, fail_after_steps=1)
    n = 400
    path = oracle.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])
    srv = Server(backend=pool, iters_per_step=1)
    futs = [srv.submit(*path) for _ in range(5)]
    for f in futs:
        with pytest.raises(RuntimeError):
            f.result(timeout=30)
    srv._thread.join(timeout=10)
    assert not srv._thread.is_alive()


def test_concurrent_submitters():
    from paper_1910_05971_gb300.serve import Server
    graphs = _graphs(40, seed=5)
    pool = FakePool(budget=50_000, max_slots=6)
    results = {}
    with Server(backend=pool, iters_per_step=2) as srv:
        def client(idx):
            for i in range(idx, len(graphs), 4):
                results[i] = srv.submit(*graphs[i]).result(timeout=60)
        ths = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    for i, (rp, ci) in enumerate(graphs):
        f, it, _, _ = oracle.fastsv(rp, ci)
        assert np.array_equal(results[i][0], f) and results[i][1] == it


def test_preemption_lets_small_requests_pass_and_resumes_exactly():
    """A long-running graph fills the pool; with preemption on, requests that
    cannot fit make the server checkpoint it, run one of them, and resume it:
    every result equals solving alone, and a small request no longer waits for
    the long graph to finish."""
    from paper_1910_05971_gb300.serve import Server
    n = 400
    long_path = oracle.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])  # ~log-many iterations, big
    smalls = _graphs(6, seed=5)
    pool_bytes = FakePool(0, 1).bytes_for(n, len(long_path[1]))

    def run(preempt):
        backend = FakePool(pool_bytes + 64, 8, step_delay=0.01)
        srv = Server(backend=backend, preempt_after_steps=preempt)
        futs = [srv.submit(*long_path)]
        # let the long graph start (it needs 9 steps), then queue the small ones
        t0 = time.time()
        while backend.steps < 1 and time.time() - t0 < 30:
            time.sleep(0.0005)
        futs += [srv.submit(rp, ci) for rp, ci in smalls]
        res = [f.result(timeout=60) for f in futs]
        srv.close()
        return res, backend, srv

    def is_long(r):
        return len(r.rp) == n + 1

    for preempt in (0, 2):
        res, backend, srv = run(preempt)
        for (rp, ci), (lab, it) in zip([long_path] + smalls, res):
            f, it_ref, _, _ = oracle.fastsv(rp, ci)
            assert np.array_equal(lab, f) and it == it_ref
        if preempt:
            assert backend.evicted >= 1 and srv.evictions == backend.evicted
            # a small request finished before the long graph instead of waiting for it
            assert not is_long(srv.completed[0])
        else:
            assert backend.evicted == 0
            assert is_long(srv.completed[0])

"""Pins for the CPU oracle (no GPU).

Each oracle function is checked against something other than itself:
hand-worked traces of Algorithm 2 (tests/golden), breadth-first search on
every graph with at most five vertices, closed forms, scipy's connected
components (a library routine for the same partition), Lemma 1 and the
early-termination theorem of Appendix A, and the equivalence of the
Algorithm 2 and Algorithm 3 formulations.  The mutant tests plant plausible
mistakes in the oracle source and show that these pins catch each of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "alg2_hand_traces.json")
FORMS = ("alg2", "alg3", "omp")


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


def _random_graph(n, m_und, rng, self_loops=False, dups=False):
    edges = []
    for _ in range(m_und):
        u, v = int(rng.integers(n)), int(rng.integers(n))
        if u == v and not self_loops:
            continue
        edges.append((u, v))
    if not dups:
        edges = sorted({(min(u, v), max(u, v)) for u, v in edges})
    return oracle.csr_from_edges(n, edges)


# ---------------------------------------------------------------------------
# hand-worked traces (Algorithm 2 by hand)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_traces(case, form):
    rp, ci = oracle.csr_from_edges(case["n"], case["edges"])
    f, it, conv, changed = oracle.fastsv(rp, ci, form=form)
    assert it == case["iterations"]
    assert conv
    assert changed.tolist() == case["changed"]
    assert f.tolist() == case["labels"]
    for k, f_exp in enumerate(case["f_after"], start=1):
        fk, itk, _, _ = oracle.fastsv(rp, ci, max_iters=k, form=form)
        assert itk == k
        assert fk.tolist() == f_exp, f"after iteration {k}"


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_traces_single_step(case):
    """oracle.iteration (one loop body) reproduces the same per-iteration f."""
    rp, ci = oracle.csr_from_edges(case["n"], case["edges"])
    f = np.arange(case["n"], dtype=np.int32)
    for f_exp, ch in zip(case["f_after"], case["changed"]):
        assert oracle.iteration(rp, ci, f) == ch
        assert f.tolist() == f_exp


# ---------------------------------------------------------------------------
# exhaustive: every graph with at most five vertices
# ---------------------------------------------------------------------------

def _all_graphs(max_n=5):
    for n in range(0, max_n + 1):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            yield n, [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


def test_bfs_pins_by_hand():
    rp, ci = oracle.csr_from_edges(6, [(1, 4), (4, 2), (3, 5)])
    assert oracle.bfs(rp, ci).tolist() == [0, 1, 1, 3, 1, 3]
    rp, ci = oracle.csr_from_edges(4, [])
    assert oracle.bfs(rp, ci).tolist() == [0, 1, 2, 3]
    rp, ci = oracle.csr_from_edges(5, [(4, 3), (3, 2)])
    assert oracle.bfs(rp, ci).tolist() == [0, 1, 2, 2, 2]


def test_exhaustive_small_graphs():
    count = 0
    for n, edges in _all_graphs(5):
        rp, ci = oracle.csr_from_edges(n, edges)
        ref = oracle.bfs(rp, ci)
        assert np.array_equal(oracle.uf(rp, ci), ref)
        res = [oracle.fastsv(rp, ci, form=form) for form in FORMS]
        for f, it, conv, ch in res:
            assert conv
            assert np.array_equal(f, ref), (n, edges)
        # the three formulations agree on the iteration sequence
        assert res[0][1] == res[1][1] == res[2][1]
        assert np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][3], res[2][3])
        if n > 0:
            assert res[0][1] >= 1
        count += 1
    assert count == 1 + 1 + 2 + 8 + 64 + 1024


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def test_closed_forms():
    n = 200
    rp, ci = oracle.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])           # path
    assert (oracle.fastsv(rp, ci)[0] == 0).all()
    rp, ci = oracle.csr_from_edges(n, [(0, i) for i in range(1, n)])                 # star, centre 0
    f, it, _, _ = oracle.fastsv(rp, ci)
    assert (f == 0).all() and it == 2
    rp, ci = oracle.csr_from_edges(n, [(n - 1, i) for i in range(n - 1)])            # star, centre n-1
    f, it, _, _ = oracle.fastsv(rp, ci)
    assert (f == 0).all() and it == 3
    k = 9
    rp, ci = oracle.csr_from_edges(k, list(itertools.combinations(range(k), 2)))     # clique
    f, it, _, _ = oracle.fastsv(rp, ci)
    assert (f == 0).all() and it == 2
    rp, ci = oracle.csr_from_edges(50, [])                                            # isolated vertices
    f, it, _, _ = oracle.fastsv(rp, ci)
    assert f.tolist() == list(range(50)) and it == 1


def test_closed_forms_lattice():
    side, extra = 40, 17
    rp, ci = graphgen.grid(side, 1.0, extra, seed=2)                                  # every edge kept
    for form in FORMS:
        f = oracle.fastsv(rp, ci, form=form)[0]
        assert (f[: side * side] == 0).all()
        assert f[side * side:].tolist() == list(range(side * side, side * side + extra))
    rp, ci = graphgen.grid(side, 0.0, extra, seed=2)                                  # no edge kept
    f, it, _, _ = oracle.fastsv(rp, ci)
    assert f.tolist() == list(range(side * side + extra)) and it == 1


def test_labels_match_scipy_partition():
    """scipy.sparse.csgraph.connected_components is an independent library
    routine for the same partition; the min-id labelling is then fixed."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    rp, ci = graphgen.rmat(12, 4, seed=11)
    n = len(rp) - 1
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    ncomp, comp = csgraph.connected_components(A, directed=False)
    expect = np.full(ncomp, n, dtype=np.int64)
    np.minimum.at(expect, comp, np.arange(n))
    expect = expect[comp]
    assert np.array_equal(oracle.uf(rp, ci), expect)
    for form in FORMS:
        assert np.array_equal(oracle.fastsv(rp, ci, form=form)[0], expect)


# ---------------------------------------------------------------------------
# Lemma 1, the early-termination theorem, star shape at termination
# ---------------------------------------------------------------------------

def _graphs_for_invariants():
    rng = np.random.default_rng(7)
    out = [graphgen.rmat(10, 4, seed=3, permute=True), graphgen.grid(20, 0.5, 5, seed=9)]
    for n, m in [(60, 40), (300, 200), (300, 600), (1000, 700)]:
        out.append(_random_graph(n, m, rng))
    return out


def test_lemma1_and_monotone():
    """Appendix A, Lemma 1: f[u] <= u at all times; f and f[f] never increase."""
    for rp, ci in _graphs_for_invariants():
        n = len(rp) - 1
        f = np.arange(n, dtype=np.int32)
        gf = f[f]
        while True:
            prev_f, prev_gf = f.copy(), gf.copy()
            ch = oracle.iteration(rp, ci, f)
            gf = f[f]
            assert (f <= np.arange(n)).all()
            assert (f <= prev_f).all()
            assert (gf <= prev_gf).all()
            assert ch == int((gf != prev_gf).sum())
            if ch == 0:
                break


def test_early_termination_theorem():
    """Appendix A, Theorem: once f[f] is unchanged, f never changes again; at
    that point every tree is a star and f is the component minimum."""
    for rp, ci in _graphs_for_invariants():
        f, it, conv, _ = oracle.fastsv(rp, ci)
        assert conv
        assert np.array_equal(f[f], f)                       # stars
        assert np.array_equal(f, oracle.uf(rp, ci))
        g = f.copy()
        for _ in range(3):
            assert oracle.iteration(rp, ci, g) == 0
            assert np.array_equal(g, f)


def test_self_loops_and_duplicates_are_no_ops():
    rng = np.random.default_rng(3)
    for n, m in [(100, 80), (400, 500)]:
        edges = [(int(rng.integers(n)), int(rng.integers(n))) for _ in range(m)]
        clean = sorted({(min(u, v), max(u, v)) for u, v in edges if u != v})
        noisy = clean + clean[: len(clean) // 2] + [(i, i) for i in range(0, n, 3)]
        a = oracle.fastsv(*oracle.csr_from_edges(n, clean))
        b = oracle.fastsv(*oracle.csr_from_edges(n, noisy))
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[3], b[3])


# ---------------------------------------------------------------------------
# random sweep and the small named workload
# ---------------------------------------------------------------------------

def test_random_sweep_forms_agree():
    rng = np.random.default_rng(2024)
    for trial in range(40):
        n = int(rng.integers(1, 400))
        m = int(rng.integers(0, 3 * n))
        rp, ci = _random_graph(n, m, rng)
        ref = oracle.uf(rp, ci)
        res = [oracle.fastsv(rp, ci, form=form) for form in FORMS]
        for f, it, conv, ch in res:
            assert np.array_equal(f, ref)
        assert res[0][1] == res[1][1] == res[2][1]
        assert np.array_equal(res[0][3], res[1][3]) and np.array_equal(res[0][3], res[2][3])


def test_rmat_s16_oracle():
    rp, ci = graphgen.rmat_s16()
    ref = oracle.uf(rp, ci)
    f2, it2, conv2, ch2 = oracle.fastsv(rp, ci, form="alg2")
    f3, it3, conv3, ch3 = oracle.fastsv(rp, ci, form="alg3")
    fo, ito, convo, cho = oracle.fastsv(rp, ci, form="omp", nthreads=4)
    assert conv2 and conv3 and convo
    assert np.array_equal(f2, ref) and np.array_equal(f3, ref) and np.array_equal(fo, ref)
    assert it2 == it3 == ito
    assert np.array_equal(ch2, ch3) and np.array_equal(ch2, cho)
    # Section 3.4 reports 5 to 10 iterations on real graphs: a sanity range, not a pin
    assert 2 <= it2 <= 30


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by the pins above
# ---------------------------------------------------------------------------

def _pins_pass(mutant: int) -> bool:
    try:
        for case in _cases():
            rp, ci = oracle.csr_from_edges(case["n"], case["edges"])
            f, it, conv, changed = oracle.fastsv(rp, ci, mutant=mutant)
            if it != case["iterations"] or changed.tolist() != case["changed"] or f.tolist() != case["labels"]:
                return False
            for k, f_exp in enumerate(case["f_after"], start=1):
                if oracle.fastsv(rp, ci, max_iters=k, mutant=mutant)[0].tolist() != f_exp:
                    return False
        for n, edges in _all_graphs(4):
            rp, ci = oracle.csr_from_edges(n, edges)
            f, it, conv, _ = oracle.fastsv(rp, ci, mutant=mutant, max_iters=64)
            if not conv or not np.array_equal(f, oracle.bfs(rp, ci)):
                return False
    except Exception:
        return False
    return True


def test_unmutated_oracle_passes_pins():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_planted_mistake_is_caught(mutant):
    assert not _pins_pass(mutant)

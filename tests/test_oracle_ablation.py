"""Pins for the oracle's convergence ablation sv1..sv5 (no GPU).

sv1 is the simplified SV algorithm (Algorithm 1, Section 2.4); sv2..sv5 add grandparent
hooking (Section 3.1), stochastic hooking (3.2), aggressive hooking with
Algorithm 2's single-pass body (3.3) and early termination (3.4) one at a
time, so sv5 is Algorithm 2.  Each variant is checked against hand-worked
traces (tests/golden/sv_ablation_hand_traces.json), against breadth-first
search on every graph with at most five vertices, against the invariants the
paper proves for every variant (f[u] <= u, f never increases, stars at
termination), and against the early-termination lemma of Section 3.4
(sv4 and sv5 share their iterations and differ by at most the one extra
iteration that sv4 needs to see f unchanged).  Planted mistakes in the
variant code must fail these pins.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sv_ablation_hand_traces.json")
VARIANTS = ("sv1", "sv2", "sv3", "sv4", "sv5")


def _cases():
    with open(GOLDEN) as fh:
        return json.load(fh)["cases"]


def _all_graphs(nmax):
    for n in range(nmax + 1):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            yield n, [pairs[i] for i in range(len(pairs)) if mask >> i & 1]


def _random_graphs(seed=11, count=30):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(2, 300))
        m = int(rng.integers(0, 2 * n))
        edges = sorted({(min(u, v), max(u, v)) for u, v in
                        ((int(rng.integers(n)), int(rng.integers(n))) for _ in range(m)) if u != v})
        out.append(oracle.csr_from_edges(n, edges))
    return out


def _steps(rp, ci, variant, k, mutant=0):
    """f after each of the first k iterations, via the one-iteration entry point."""
    n = len(rp) - 1
    f = np.arange(n, dtype=np.int32)
    out = []
    for _ in range(k):
        if variant == "sv5":
            oracle.iteration(rp, ci, f, mutant=mutant)
        else:
            oracle.sv_iteration(rp, ci, f, int(variant[2]), mutant=mutant)
        out.append(f.tolist())
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("variant", VARIANTS)
def test_hand_traces(case, variant):
    if variant not in case["variants"]:
        pytest.skip("no hand trace for this variant")
    exp = case["variants"][variant]
    rp, ci = oracle.csr_from_edges(case["n"], case["edges"])
    f, it, conv, changed = oracle.fastsv(rp, ci, form=variant)
    assert conv
    assert it == exp["iterations"]
    assert changed.tolist() == exp["changed"]
    assert f.tolist() == case["labels"]
    assert _steps(rp, ci, variant, len(exp["f_after"])) == exp["f_after"]
    for k, f_exp in enumerate(exp["f_after"], start=1):
        fk, itk, _, _ = oracle.fastsv(rp, ci, max_iters=k, form=variant)
        assert itk == k and fk.tolist() == f_exp


def test_exhaustive_small_graphs():
    """Every variant labels every graph of at most five vertices with its
    component minima (Algorithm 1's correctness, and Algorithm 2's)."""
    for n, edges in _all_graphs(5):
        rp, ci = oracle.csr_from_edges(n, edges)
        ref = oracle.bfs(rp, ci)
        for v in VARIANTS:
            f, it, conv, _ = oracle.fastsv(rp, ci, form=v, max_iters=64)
            assert conv and np.array_equal(f, ref), (v, n, edges)


def test_invariants_every_iteration():
    """f[u] <= u and f never increases, for every variant and iteration; at
    termination every tree is a star (f[f] == f)."""
    for rp, ci in _random_graphs():
        n = len(rp) - 1
        for v in (1, 2, 3, 4):
            f = np.arange(n, dtype=np.int32)
            for _ in range(4 * n + 4):
                prev = f.copy()
                ch = oracle.sv_iteration(rp, ci, f, v)
                assert (f <= np.arange(n)).all() and (f <= prev).all()
                assert ch == int((f != prev).sum())
                if ch == 0:
                    break
            assert ch == 0
            assert np.array_equal(f[f], f)
            assert np.array_equal(f, oracle.uf(rp, ci))


def test_sv4_is_algorithm2_without_early_termination():
    """sv4 runs Algorithm 2's iterations and stops one iteration later at most
    (Section 3.4: once f[f] is unchanged, f does not change afterwards)."""
    graphs = _random_graphs(seed=12) + [oracle.csr_from_edges(n, e) for n, e in _all_graphs(4)]
    extra = 0
    for rp, ci in graphs:
        f4, it4, c4, _ = oracle.fastsv(rp, ci, form="sv4")
        f5, it5, c5, _ = oracle.fastsv(rp, ci, form="sv5")
        assert c4 and c5 and np.array_equal(f4, f5)
        assert it5 <= it4 <= it5 + 1
        extra += it4 - it5
        k = min(it4, it5)
        assert _steps(rp, ci, "sv4", k) == _steps(rp, ci, "sv5", k)
    assert extra > 0  # the early termination does save iterations on some graphs


def test_variants_agree_in_first_iteration():
    """From f = identity every vertex is a root and f = f[f], so sv1, sv2 and
    sv3 take the same first iteration."""
    for rp, ci in _random_graphs(seed=13, count=10):
        a, b, c = (_steps(rp, ci, v, 1) for v in ("sv1", "sv2", "sv3"))
        assert a == b == c


def _pins_pass(mutant: int) -> bool:
    try:
        for case in _cases():
            rp, ci = oracle.csr_from_edges(case["n"], case["edges"])
            for v, exp in case["variants"].items():
                f, it, conv, changed = oracle.fastsv(rp, ci, form=v, mutant=mutant, max_iters=64)
                if it != exp["iterations"] or changed.tolist() != exp["changed"] or f.tolist() != case["labels"]:
                    return False
                if _steps(rp, ci, v, len(exp["f_after"]), mutant=mutant) != exp["f_after"]:
                    return False
        for n, edges in _all_graphs(4):
            rp, ci = oracle.csr_from_edges(n, edges)
            for v in VARIANTS:
                f, it, conv, _ = oracle.fastsv(rp, ci, form=v, mutant=mutant, max_iters=64)
                if not conv or not np.array_equal(f, oracle.bfs(rp, ci)):
                    return False
    except Exception:
        return False
    return True


def test_unmutated_oracle_passes_pins():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", [6, 7])
def test_planted_mistake_is_caught(mutant):
    """6: the root test of sv1/sv2 dropped; 7: the shortcut of Algorithm 1
    taken from the pointer graph before hooking."""
    assert not _pins_pass(mutant)

"""Host-side tests of the tuning cache: shape-class keys and the cache
file's round trip (no GPU needed)."""
import os

import paper_1910_05971_gb300 as fsv
from paper_1910_05971_gb300 import tune


def test_tune_keys():
    # R-MAT scale 26: 2^26 vertices, 31.35 entries per vertex (log2 = 4.97 -> 10 half-octaves)
    assert fsv.fastsv_tune_key(fsv.TUNE_SINGLE, 1 << 26, 2103860902, 1, 64) == "single n26 d10 r64"
    assert fsv.fastsv_tune_key(fsv.TUNE_SINGLE, 65536, 1818976, 1, 32) == "single n16 d10 r32"
    assert fsv.fastsv_tune_key(fsv.TUNE_SINGLE, 100, 0, 1, 32) == "single n7 d-99 r32"
    # 4096 graphs, 108e6 vertices in all (26,367 per graph), 10.2 entries per vertex
    assert fsv.fastsv_tune_key(fsv.TUNE_BATCHED, 108_000_000, 1_100_000_000, 4096, 32) == "batched g12 n15 d7"


def test_cache_round_trip(tmp_path):
    p = os.path.join(tmp_path, "cache.txt")
    entries = {"single n26 d10 r64": dict(k2_items=8, k2_threads=256, col_blocks=16, sparse_div=2,
                                          batch_sparse_div=0),
               "batched g12 n15 d7": dict(k2_items=4, k2_threads=64, col_blocks=0, sparse_div=2,
                                          batch_sparse_div=16)}
    tune.write_cache(p, entries, {"single n26 d10 r64": "a note"})
    assert tune.read_cache(p) == entries
    # a later line for a key replaces an earlier one; malformed lines are skipped
    with open(p, "a") as fh:
        fh.write("single n26 d10 r64 = 16 64 8 0 0\nnot a line\nsingle n1 = 1 2\n")
    got = tune.read_cache(p)
    assert got["single n26 d10 r64"] == dict(k2_items=16, k2_threads=64, col_blocks=8, sparse_div=0,
                                             batch_sparse_div=0)
    assert "single n1" not in got
    assert tune.read_cache(os.path.join(tmp_path, "missing.txt")) == {}


def test_coordinate_descent_picks_the_fastest():
    # a synthetic cost: col_blocks 8 and tile (64, 16) are best, sparse_div irrelevant
    def cost(s):
        return (abs(s["col_blocks"] - 8) + (0 if (s["k2_threads"], s["k2_items"]) == (64, 16) else 3)
                + 0.1 * s["sparse_div"])
    knobs = [[dict(col_blocks=c) for c in (1, 4, 8, 16)],
             [dict(k2_threads=t, k2_items=i) for t, i in tune.TILE_SHAPES],
             [dict(sparse_div=d) for d in (0, 2, 4)]]
    best, ms, table = tune._descend(cost, knobs, tune.DEFAULTS)
    assert (best["col_blocks"], best["k2_threads"], best["k2_items"], best["sparse_div"]) == (8, 64, 16, 0)
    assert ms == cost(best) and len(table) <= 1 + 4 + len(tune.TILE_SHAPES) + 3

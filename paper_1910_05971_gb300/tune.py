"""Autotuner of libfastsv's kernel choices; writes the tuning cache.

The paper leaves the switch between the SpMV and the sparse SpMSpV to tuning
(Section 4.2 gives no threshold), and the best merge-path tile shape and
number of column blocks depend on the graph's size and density.  For one
graph (or one batch of graphs) the tuner times candidate settings of

    k2_items, k2_threads   merge-path items per thread and CTA size of the SpMV
    col_blocks             column blocks of a large graph's SpMV (single graphs)
    sparse_div             single graphs: push when the changed vertices' degree
                           sum is <= m / sparse_div (0 = never)
    batch_sparse_div       batched calls: the same per graph

on the device (one untimed solve, then CUDA events around ``steps`` solves
per candidate), checks that every candidate returns the same labels and
iteration count as the first (the arithmetic is exact, so they must), and
records the fastest under the call's shape-class key (``fastsv_tune_key``:
log2 of the vertex count, half-octaves of the entries per vertex, row-pointer
width; for batches the graph count and mean graph size).  The search is a
coordinate descent from the library's defaults, one knob at a time.

    python -m paper_1910_05971_gb300.tune --workloads rmat_s26_perm,er_batch \\
        --cache paper_1910_05971_gb300/tune_cache.txt

Cache lines:  ``<key> = <k2_items> <k2_threads> <col_blocks> <sparse_div> <batch_sparse_div>``.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import _lib

DEFAULTS = dict(k2_items=8, k2_threads=256, col_blocks=0, sparse_div=2, batch_sparse_div=0)
FIELDS = ("k2_items", "k2_threads", "col_blocks", "sparse_div", "batch_sparse_div")
TILE_SHAPES = [(256, 8), (256, 4), (256, 16), (64, 8), (64, 16)]


def _log(*a):
    print(*a, file=sys.stderr, flush=True)


def read_cache(path: str) -> dict:
    """{key: settings} of a cache file (later lines win); {} if absent."""
    out = {}
    if not path or not os.path.exists(path):
        return out
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0]
            if "=" not in line:
                continue
            key, vals = line.split("=", 1)
            parts = vals.split()
            if len(parts) != 5:
                continue
            out[key.strip()] = dict(zip(FIELDS, (int(x) for x in parts)))
    return out


def write_cache(path: str, entries: dict, notes: dict | None = None):
    """Write {key: settings} as a cache file (one line per key, sorted)."""
    lines = ["# libfastsv tuning cache: <shape key> = k2_items k2_threads col_blocks sparse_div batch_sparse_div"]
    for key in sorted(entries):
        s = entries[key]
        note = f"  # {notes[key]}" if notes and key in notes else ""
        lines.append(f"{key} = " + " ".join(str(int(s[f])) for f in FIELDS) + note)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    os.replace(tmp, path)


def _time_single(rp_d, ci_d, bits, settings, steps):
    import torch
    from . import FastSV
    stream = torch.cuda.current_stream()
    with FastSV(rowptr_bits=bits, tune_cache=None, **settings) as s:
        lab = s.cc(rp_d, ci_d)
        st = s.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            s.cc(rp_d, ci_d, lab, check_status=False)
        e1.record(stream)
        torch.cuda.synchronize()
        s.check_last()
        return e0.elapsed_time(e1) / steps, lab.clone(), st["iterations"], st


def _time_batched(d, settings, steps):
    import torch
    from . import FastSV
    stream = torch.cuda.current_stream()
    with FastSV(rowptr_bits=32, tune_cache=None, **settings) as s:
        lab, it = s.cc_batched(d["vtx_off"], d["edge_off"], d["row_ptr"], d["col_idx"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            s.cc_batched(d["vtx_off"], d["edge_off"], d["row_ptr"], d["col_idx"], lab, it, check_status=False)
        e1.record(stream)
        torch.cuda.synchronize()
        s.check_last()
        return e0.elapsed_time(e1) / steps, lab.clone(), it.clone(), None


def _descend(measure, knobs, start):
    """Coordinate descent: for every knob in turn, time its candidates with
    the others fixed at the best so far.  measure(settings) -> ms."""
    best = dict(start)
    table = {}

    def run(s):
        key = tuple(s[f] for f in FIELDS)
        if key not in table:
            table[key] = measure(s)
        return table[key]

    best_ms = run(best)
    for cands in knobs:
        for c in cands:
            s = dict(best)
            s.update(c)
            ms = run(s)
            if ms < best_ms:
                best, best_ms = s, ms
    return best, best_ms, table


def tune_single(rp_d, ci_d, bits: int = 64, steps: int = 3, l2_bytes: int = 129 << 20):
    """Tune one graph (device CSR).  Returns a dict with its key, the best
    settings, their time, the default settings' time and every timing."""
    n, m = rp_d.numel() - 1, ci_d.numel()
    key = _lib.fastsv_tune_key(_lib.TUNE_SINGLE, n, m, 1, bits)
    ref = {}

    def measure(s):
        ms, lab, it, _ = _time_single(rp_d, ci_d, bits, s, steps)
        if not ref:
            ref.update(lab=lab, it=it)
        elif not (it == ref["it"] and bool((lab == ref["lab"]).all())):
            raise AssertionError(f"tuning candidate {s} changed the labels or iterations")
        _log(f"[tune] {key} {s} {ms:.3f} ms")
        return ms

    knobs = []
    if 4 * n >= l2_bytes and m >= 8 * n:
        knobs.append([dict(col_blocks=c) for c in (1, 4, 8, 16, 32)])
    knobs.append([dict(k2_threads=t, k2_items=i) for t, i in TILE_SHAPES])
    knobs.append([dict(sparse_div=d) for d in (0, 2, 4, 8)])
    best, best_ms, table = _descend(measure, knobs, DEFAULTS)
    return dict(key=key, best=best, best_ms=best_ms, default_ms=table[tuple(DEFAULTS[f] for f in FIELDS)],
                candidates=len(table))


def tune_batched(d, steps: int = 3):
    """Tune one batch (dict of device tensors vtx_off, edge_off, row_ptr, col_idx)."""
    G = d["vtx_off"].numel() - 1
    N, M = int(d["vtx_off"][-1].item()), int(d["edge_off"][-1].item())
    key = _lib.fastsv_tune_key(_lib.TUNE_BATCHED, N, M, G, 32)
    ref = {}

    def measure(s):
        ms, lab, it, _ = _time_batched(d, s, steps)
        if not ref:
            ref.update(lab=lab, it=it)
        elif not (bool((it == ref["it"]).all()) and bool((lab == ref["lab"]).all())):
            raise AssertionError(f"tuning candidate {s} changed the labels or iterations")
        _log(f"[tune] {key} {s} {ms:.3f} ms")
        return ms

    knobs = [[dict(k2_threads=t, k2_items=i) for t, i in TILE_SHAPES],
             [dict(batch_sparse_div=b) for b in (0, 4, 16)]]
    best, best_ms, table = _descend(measure, knobs, DEFAULTS)
    return dict(key=key, best=best, best_ms=best_ms, default_ms=table[tuple(DEFAULTS[f] for f in FIELDS)],
                candidates=len(table))


def main(argv=None):
    import torch

    import graphgen

    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workloads", default="rmat_s26_perm,grid_4096_p055_iso1M,er_batch")
    ap.add_argument("--cache", required=True, help="cache file to update")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--graphs", type=int, default=4096, help="er_batch: number of graphs")
    args = ap.parse_args(argv)
    torch.cuda.init()
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    entries = read_cache(args.cache)
    notes = {}
    for name in args.workloads.split(","):
        t0 = time.time()
        if name == "er_batch":
            b = graphgen.er_batch(args.graphs, seed=4)
            d = {k: torch.from_numpy(getattr(b, k)).cuda() for k in ("vtx_off", "edge_off", "row_ptr", "col_idx")}
            res = tune_batched(d, args.steps)
            del d
        else:
            rp, ci = graphgen.WORKLOADS[name]()
            bits = 64 if len(ci) > np.iinfo(np.int32).max // 2 else 32
            rp_d = torch.from_numpy(rp.astype(np.int64 if bits == 64 else np.int32)).cuda()
            ci_d = torch.from_numpy(ci).cuda()
            del rp, ci
            res = tune_single(rp_d, ci_d, bits, args.steps, l2)
            del rp_d, ci_d
        torch.cuda.empty_cache()
        entries[res["key"]] = res["best"]
        notes[res["key"]] = f"{name}: {res['best_ms']:.3f} ms tuned, {res['default_ms']:.3f} ms default"
        res["workload"] = name
        res["seconds"] = time.time() - t0
        print(json.dumps(res), flush=True)
        write_cache(args.cache, entries, notes)


if __name__ == "__main__":
    main()

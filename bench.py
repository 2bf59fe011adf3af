#!/usr/bin/env python3
"""Benchmark: FastSV connected components on one GB300 (or N replicas).

One step = one complete FastSV solve (set-up + every iteration until f[f]
stops changing) of the workload through the C ABI.  Default workload: R-MAT
scale 26, edge factor 16, ids permuted (67,108,864 vertices, ~2.1e9 directed
CSR entries, int64 row_ptr).  The metric is directed CSR entries per second
of the whole solve (GTEPS = 1e9 entries/s), inputs resident in HBM.

Also reported:
  e2e          the same metric through fastsv_cc_host from pinned host
               buffers: the host-to-device copy of row_ptr/col_idx and the
               copy back of the labels are inside every timed step;
  roofline     the SpMV kernel (k2_spmv, the largest share of device time):
               counted algorithmic bytes per launch / its average duration
               (CUDA events on its stream, host-loop pass over the same
               steps, full-SpMV iterations only) against the measured HBM
               copy bandwidth;
  cpu_baseline the CPU oracle (OpenMP Algorithm 2) on the same graph on the
               host cores.

--impl reference times the CPU oracle as the reference arm.
Multi-GPU (torchrun): every rank solves its own replica of the workload
(the single-graph solve does not shard); value = all ranks' entries / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
from paper_1910_05971_gb300.clocks import ClockSampler  # noqa: E402,F401

WORKLOADS = {
    "rmat_s26_perm": dict(desc="R-MAT scale 26, edge factor 16, a/b/c=.57/.19/.19, ids permuted, seed 3",
                          bits=64),
    "rmat_s16": dict(desc="R-MAT scale 16, edge factor 16, seed 1", bits=32),
    "rmat_s25_ef8_perm": dict(desc="R-MAT scale 25, edge factor 8, ids permuted, seed 3 (profiling case)",
                              bits=64),
    "grid_4096_p055_iso1M": dict(desc="4096x4096 lattice, p=0.55, +1M isolated, seed 2", bits=32),
}
METRIC = "CC |E|/s (GTEPS) + %HBM peak at R-MAT s26; batched graphs/s; serve p50/p99"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def kernel_source_hash() -> str:
    """Hash of the SpMV kernel's source text (k2_spmv, from its template line
    through its closing brace), so that a committed traffic figure is dropped
    once the kernel changes."""
    p = os.path.join(ROOT, "paper_1910_05971_gb300", "csrc", "fastsv_kernels.cuh")
    with open(p) as fh:
        src = fh.read()
    parts = []
    for sig in (" k2_spmv(Ctx* __restrict__ ctx, int block) {",):
        at = src.index(sig)
        start = src.rindex("template <", 0, at)
        parts.append(src[start:src.index("\n}\n", at) + 3])
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def profiled_traffic(workload: str, col_blocks=None):
    """DRAM bytes per k2_spmv launch (a full SpMV) from the committed ncu
    summary, if it was taken on the current kernel source, for this workload
    and column-block count (else None)."""
    p = os.path.join(ROOT, "profiles", "k2_spmv_traffic.txt")
    try:
        rows = {}
        with open(p) as fh:
            for line in fh:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    rows[k.strip()] = v.strip()
        if rows.get("kernel_source_sha256_16") != kernel_source_hash() or rows.get("workload") != workload:
            return None
        if col_blocks is not None and rows.get("col_blocks") != str(col_blocks):
            return None
        return float(rows["dram_bytes_per_launch"])
    except Exception:
        return None


def make_graph(workload: str):
    t0 = time.time()
    rp, ci = graphgen.WORKLOADS[workload]()
    log(f"[bench] generated {workload}: n={len(rp) - 1} m={len(ci)} in {time.time() - t0:.1f}s")
    return rp, ci


def cpu_oracle_time(rp, ci, max_seconds: float = 30.0):
    """Time the CPU oracle (OpenMP Algorithm 2, all host threads) on the
    graph.  The sample is the full solve when it fits the time bound; else a
    prefix of iterations, scaled by the iterations the solve needs."""
    import oracle
    nthreads = os.cpu_count() or 1
    t0 = time.time()
    f, it1, conv1, _ = oracle.fastsv(rp, ci, form="omp", nthreads=nthreads, max_iters=1)
    t_first = time.time() - t0
    if conv1:
        return dict(seconds=t_first, iterations=1, sample="full solve (1 iteration)", cores=nthreads)
    if t_first * 8 <= max_seconds:
        t0 = time.time()
        f, it, conv, _ = oracle.fastsv(rp, ci, form="omp", nthreads=nthreads)
        return dict(seconds=time.time() - t0, iterations=it, sample=f"full solve ({it} iterations)",
                    cores=nthreads)
    return dict(seconds=t_first, iterations=1, sample="first iteration only (time per iteration)",
                cores=nthreads, per_iteration=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fastsv", choices=["fastsv", "reference"])
    ap.add_argument("--workload", default="rmat_s26_perm", choices=sorted(WORKLOADS))
    ap.add_argument("--k2-items", type=int, default=None,
                    help="SpMV items per thread (default: the library's choice, or the tuning cache's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--col-blocks", type=int, default=None,
                    help="column blocks (default: the library's choice, or the tuning cache's)")
    ap.add_argument("--mode", default="single", choices=["single", "batched", "serve", "variants"],
                    help="single: one large graph (default, the headline); batched: 4096 ER graphs in one "
                         "launch vs per-graph launches; serve: replay of the request trace; variants: "
                         "iterations and time of the convergence ablation sv1..sv5 and the asynchronous mode")
    ap.add_argument("--variant-workloads", default="rmat_s16,grid_4096_p055_iso1M,rmat_s26_perm",
                    help="variants mode: comma-separated workloads")
    ap.add_argument("--graphs", type=int, default=4096, help="batched mode: number of graphs")
    ap.add_argument("--requests", type=int, default=4096, help="serve: arrivals of the trace replayed")
    ap.add_argument("--distinct", type=int, default=256,
                    help="serve: distinct request graphs materialised (arrival i carries graph i mod this)")
    ap.add_argument("--no-batched", action="store_true", help="single mode: leave out the batched measurement")
    ap.add_argument("--no-serve", action="store_true", help="single mode: leave out the serving measurement")
    ap.add_argument("--batch-sparse-div", type=int, default=None,
                    help="batched/serve modes: per-graph sparse iterations threshold (0 = off)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    peaks, peak_src = measured_peaks()
    args.peak_gbs, args.peak_source = float(peaks["hbm_gbs"]), f"{peak_src} hbm_gbs"
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "batched":
        from paper_1910_05971_gb300 import benchmarks as bench_modes
        return bench_modes.run_batched(args, rank, world, local_rank)
    if args.mode == "serve":
        from paper_1910_05971_gb300 import benchmarks as bench_modes
        return bench_modes.run_serve(args, rank, world, local_rank)
    if args.mode == "variants":
        from paper_1910_05971_gb300 import benchmarks as bench_modes
        return bench_modes.run_variants(args, rank, world, local_rank)

    import torch
    import paper_1910_05971_gb300 as fsv

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    wl = WORKLOADS[args.workload]
    bits = wl["bits"]
    rp, ci = make_graph(args.workload)
    n, m = len(rp) - 1, len(ci)
    rp_dev = torch.from_numpy(rp.astype(np.int64 if bits == 64 else np.int32)).cuda()
    ci_dev = torch.from_numpy(ci).cuda()
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    solver = fsv.FastSV(rowptr_bits=bits, k2_items=args.k2_items, col_blocks=args.col_blocks)
    for _ in range(args.warmup):
        solver.cc(rp_dev, ci_dev, labels)
    st = solver.stats()
    iterations = st["iterations"]
    tune_key = fsv.fastsv_tune_key(fsv.TUNE_SINGLE, n, m, 1, bits)

    # ---- timed region: K solves, inputs resident in HBM (9 GB >> 129 MB L2) ----
    def barrier():
        if dist is not None:
            dist.barrier()

    sampler = ClockSampler(local_rank)
    launches0 = solver.kernel_launches()
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        solver.cc(rp_dev, ci_dev, labels, check_status=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    solver.check_last()
    launches = solver.kernel_launches() - launches0
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * m / (ms * 1e-3) / 1e9

    # ---- the same steps with the library's hand-picked defaults (no tuning cache) ----
    hand = fsv.FastSV(rowptr_bits=bits, tune_cache=None)
    for _ in range(args.warmup):
        hand.cc(rp_dev, ci_dev, labels)
    torch.cuda.synchronize()
    eh0, eh1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eh0.record(stream)
    for _ in range(args.steps):
        hand.cc(rp_dev, ci_dev, labels, check_status=False)
    eh1.record(stream)
    torch.cuda.synchronize()
    hand.check_last()
    ms_hand = eh0.elapsed_time(eh1) / args.steps
    hand.close()
    tuning = {"key": tune_key, "tuned": bool(st["tuned"]), "ms_per_step": ms, "ms_per_step_hand_picked": ms_hand,
              "cache": "paper_1910_05971_gb300/tune_cache.txt (written by paper_1910_05971_gb300/tune.py on GB300)"}

    # ---- dominant kernel: k2_spmv durations from CUDA events (host-loop pass) ----
    prof = fsv.FastSV(rowptr_bits=bits, k2_items=args.k2_items, col_blocks=args.col_blocks, use_graph=False)
    prof.cc(rp_dev, ci_dev, labels)  # untimed: first launches of the host-loop path
    k2_ms, k3_ms, hook_ms, it_sum, dense_sum, t_sum, t_dense = 0.0, 0.0, 0.0, 0, 0, 0, 0
    for _ in range(args.steps):
        prof.cc(rp_dev, ci_dev, labels)
        sp = prof.stats()
        k2_ms += sp["ms_k2"]
        k3_ms += sp["ms_k3"]
        hook_ms += sp["ms_hook"]
        it_sum += sp["iterations"]
        dense_sum += sp["dense_iters"]
        t_sum += sp["timed_iters"]
        t_dense += sp["timed_dense_iters"]
    prof.close()
    # a column-blocked solve runs its first iteration before the host loop
    # (on the original CSR, no gathers): the averages cover the loop's
    # iterations, so k2_spmv's is that of a blocked full SpMV
    k2_avg_ms = k2_ms / max(t_dense, 1)
    k3_avg_ms = k3_ms / max(t_sum, 1)
    hook_avg_ms = hook_ms / max(t_sum, 1)
    r = 8 if bits == 64 else 4
    # counted bytes per full-SpMV launch: row pointers, column ids, one
    # gathered int32 of gf per entry, one mngf store per row
    k2_bytes = r * (n + 1) + 8 * m + 4 * n
    k3_bytes = 20 * n                                # f, gathered f[f], gf read+write, p write
    hook_bytes = 20 * n                              # mngf, gf, p reads; f read-modify-write
    peaks, peak_src = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    k2_gbs = k2_bytes / (k2_avg_ms * 1e-3) / 1e9
    # one full iteration on the counted model r(n+1) + 8m + 44n (SpMV, the
    # three hooks, grandparents + termination + snapshot)
    iter_bytes = r * (n + 1) + 8 * m + 44 * n
    iter_ms = k2_avg_ms + hook_avg_ms + k3_avg_ms
    per_iter = {"algorithmic_bytes": iter_bytes, "ms": iter_ms,
                "achieved": iter_bytes / (iter_ms * 1e-3) / 1e9,
                "frac": iter_bytes / (iter_ms * 1e-3) / 1e9 / peak,
                "frac_of_nominal_8000": iter_bytes / (iter_ms * 1e-3) / 1e9 / 8000.0,
                "model": "r(n+1) + 8m + 44n over k2_spmv + k2_hook + k3_grandparent averages"}
    traffic = profiled_traffic(args.workload, st.get("col_blocks"))

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        rp_h = torch.from_numpy(rp.astype(np.int64 if bits == 64 else np.int32)).pin_memory()
        ci_h = torch.from_numpy(ci).pin_memory()
        lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
        hsolver = fsv.FastSV(rowptr_bits=bits, k2_items=args.k2_items, col_blocks=args.col_blocks)
        # warm-up: the first device transfers out of freshly pinned pages run
        # at a fraction of the link's speed (first-touch mapping)
        for _ in range(args.warmup):
            hsolver.cc_host(rp_h, ci_h, lab_h)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            hsolver.cc_host(rp_h, ci_h, lab_h)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / args.steps
        ms_e2e = max(e0.elapsed_time(e1) / args.steps, wall * 1e3)
        if dist is not None:
            t = torch.tensor([ms_e2e], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e2e = float(t.item())
        hsolver.close()
        ok = bool(torch.equal(lab_h, labels.cpu()))
        e2e = {"value": world * m / (ms_e2e * 1e-3) / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": int(rp_h.numel() * rp_h.element_size() + ci_h.numel() * 4),
               "d2h_bytes_per_step": int(n * 4), "ms_per_step": ms_e2e, "labels_match_device_path": ok}

    solver.close()
    del rp_dev, ci_dev, labels
    torch.cuda.empty_cache()

    # ---- the other two parts of the metric: batched graphs/s, serve p50/p99 ----
    from paper_1910_05971_gb300 import benchmarks as bench_modes
    batched = serve = None
    if not args.no_batched:
        try:
            batched = bench_modes.batched_measure(args.graphs, max(3, args.steps // 2), args.warmup, args.k2_items,
                                                  args.batch_sparse_div, local_rank, dist, rank, world,
                                                  sampler=ClockSampler(local_rank), peak_gbs=args.peak_gbs,
                                                  peak_source=args.peak_source)
        except Exception as e:  # reported in the line; the headline stands on its own
            batched = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.empty_cache()
    if not args.no_serve and rank == 0:
        try:
            serve = bench_modes.serve_measure(args.requests, args.distinct, args.k2_items, args.batch_sparse_div,
                                              sampler=ClockSampler(local_rank))
        except Exception as e:
            serve = {"error": f"{type(e).__name__}: {e}"}
    # the CPU oracle last: its OpenMP threads load every host core, and the
    # batched and serving measurements depend on the host's launch latency
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c = cpu_oracle_time(rp, ci)
        if c.get("per_iteration"):
            secs = c["seconds"] * iterations
            sample = c["sample"] + f", scaled by the {iterations} iterations of the solve"
        else:
            secs = c["seconds"]
            sample = c["sample"]
        cpu = {"value": m / secs / 1e9, "unit": "GTEPS", "cores": c["cores"], "kind": "oracle",
               "sample": f"{args.workload}: {sample}, OpenMP Algorithm 2 on the host cores",
               "seconds": secs}

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": value,
            "unit": "GTEPS",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "n": n, "m_directed": m,
                       "m_undirected": m // 2, "rowptr_bits": bits, "iterations": iterations,
                       "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (col_idx alone is 4m bytes), no flush",
                       "k2_items": args.k2_items, "col_blocks": st.get("col_blocks")},
            "roofline": {"bound": "hbm", "achieved": k2_gbs, "peak": peak, "unit": "GB/s",
                         "frac": k2_gbs / peak, "traffic": traffic,
                         "kernel": "k2_spmv (one launch per column block when blocked)",
                         "algorithmic_bytes_per_launch": k2_bytes,
                         "avg_launch_ms": k2_avg_ms, "peak_source": f"{peak_src} hbm_gbs",
                         "k3_grandparent": {"algorithmic_bytes_per_launch": k3_bytes, "avg_launch_ms": k3_avg_ms,
                                            "achieved": k3_bytes / (k3_avg_ms * 1e-3) / 1e9},
                         "k2_hook": {"algorithmic_bytes_per_launch": hook_bytes, "avg_launch_ms": hook_avg_ms,
                                     "achieved": hook_bytes / (hook_avg_ms * 1e-3) / 1e9},
                         "per_iteration": per_iter,
                         "dense_iterations_per_solve": dense_sum / args.steps,
                         "sparse_iterations_per_solve": (it_sum - dense_sum) / args.steps,
                         "averaged_dense_launches_per_solve": t_dense / args.steps},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "tuning": tuning,
            "batched": batched,
            "serve": serve,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle (OpenMP Algorithm 2) on the host cores,
    same workload, metric and unit; rank 0 only."""
    if rank != 0:
        return
    import oracle
    rp, ci = make_graph(args.workload)
    n, m = len(rp) - 1, len(ci)
    nthreads = os.cpu_count() or 1
    f, it, conv, _ = oracle.fastsv(rp, ci, form="omp", nthreads=nthreads, max_iters=1)
    t0 = time.time()
    oracle.fastsv(rp, ci, form="omp", nthreads=nthreads, max_iters=1)
    t_iter = time.time() - t0
    full = t_iter * 6 <= 20.0
    # the iteration count of the whole solve (oracle's own)
    if full:
        f, iters, conv, _ = oracle.fastsv(rp, ci, form="omp", nthreads=nthreads)
    else:
        iters = None
    for _ in range(max(0, args.warmup - 1)):
        if full:
            oracle.fastsv(rp, ci, form="omp", nthreads=nthreads)
    times = []
    for _ in range(args.steps):
        t0 = time.time()
        if full:
            oracle.fastsv(rp, ci, form="omp", nthreads=nthreads)
        else:
            oracle.fastsv(rp, ci, form="omp", nthreads=nthreads, max_iters=1)
        times.append(time.time() - t0)
    step = float(np.mean(times))
    if not full:
        f, iters, conv, _ = oracle.fastsv(rp, ci, form="omp", nthreads=nthreads)
        step = step * iters
        sample = f"first iteration per step, scaled by the oracle's {iters} iterations"
    else:
        sample = f"full solve per step ({iters} iterations)"
    value = m / step / 1e9
    out = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "int32", "data": "synthetic", "impl": "reference",
           "config": {"workload": args.workload, "n": n, "m_directed": m, "iterations": iters},
           "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": nthreads, "kind": "oracle",
                            "sample": f"{args.workload}: {sample}"},
           "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()

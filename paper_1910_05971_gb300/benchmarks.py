"""Batched and serving benchmark modes of bench.py.

batched  One segmented solve of G independent Erdos-Renyi graphs (one device
         loop for the whole batch, each graph stopping at its own early
         termination) against G plain per-graph fastsv_cc calls on the same
         GPU.  Both must give identical labels and iteration counts.
serve    Replay of a prefix of the request trace through the continuous-
         batching server (HBM-budget admission, slots join at iteration
         boundaries) against the same requests solved one after another with
         plain fastsv_cc_host calls in arrival order.  Latency runs from
         arrival to labels in host memory.
"""
from __future__ import annotations

import json
import sys
import threading
import time

import numpy as np


def _log(*a):
    print(*a, file=sys.stderr, flush=True)


def _clock_sampler(local_rank):
    from .clocks import ClockSampler
    return ClockSampler(local_rank)


def run_batched(args, rank, world, local_rank):
    import torch

    import graphgen
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300.replicas import batch_work, max_over_ranks, shard_graphs

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    t0 = time.time()
    full = graphgen.er_batch(args.graphs, seed=4)
    if world > 1:
        mine = shard_graphs(batch_work(full), world)[rank]
        batch = graphgen.Batch.from_graphs([full.graph(g) for g in mine])
    else:
        batch = full
    G = batch.num_graphs
    N, M = int(batch.vtx_off[-1]), int(batch.edge_off[-1])
    _log(f"[bench] batch of {G} graphs, n={N} m={M}, generated in {time.time() - t0:.1f}s")
    d = {k: torch.from_numpy(getattr(batch, k)).cuda() for k in ("vtx_off", "edge_off", "row_ptr", "col_idx")}
    stream = torch.cuda.current_stream()
    solver = fsv.FastSV(rowptr_bits=32, k2_items=args.k2_items, batch_sparse_div=args.batch_sparse_div)
    labels = torch.empty(N, dtype=torch.int32, device="cuda")
    iters = torch.empty(G, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        solver.cc_batched(d["vtx_off"], d["edge_off"], d["row_ptr"], d["col_idx"], labels, iters)
    launches0 = solver.kernel_launches()
    sampler = _clock_sampler(local_rank)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        solver.cc_batched(d["vtx_off"], d["edge_off"], d["row_ptr"], d["col_idx"], labels, iters,
                          check_status=False)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    solver.check_last()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist)
    launches = solver.kernel_launches() - launches0
    lab_b = labels.cpu().numpy()
    it_b = iters.cpu().numpy()

    # per-graph plain launches of the same kernels, one graph after another
    plain = fsv.FastSV(rowptr_bits=32, k2_items=args.k2_items)
    vo, eo = batch.vtx_off, batch.edge_off
    lab_p = torch.empty(N, dtype=torch.int32, device="cuda")
    it_p = np.zeros(G, dtype=np.int64)
    rp_all, ci_all = d["row_ptr"], d["col_idx"]

    def one_pass(record):
        for g in range(G):
            v0, v1, e0_, e1_ = int(vo[g]), int(vo[g + 1]), int(eo[g]), int(eo[g + 1])
            plain.cc(rp_all[v0 + g: v1 + g + 1], ci_all[e0_:e1_] if e1_ > e0_ else ci_all[:1],
                     lab_p[v0:v1], check_status=False)
            if record:
                it_p[g] = plain.stats()["iterations"]

    one_pass(True)  # warm-up and per-graph iteration counts
    torch.cuda.synchronize()
    t = time.perf_counter()
    one_pass(False)
    torch.cuda.synchronize()
    plain_s = max_over_ranks(time.perf_counter() - t, dist)
    same = bool(np.array_equal(lab_p.cpu().numpy(), lab_b)) and bool(np.array_equal(it_p, it_b))
    total_graphs = args.graphs if world > 1 else G
    value = total_graphs / (ms * 1e-3)
    plain.close()
    solver.close()
    if rank == 0:
        print(json.dumps({
            "metric": "batched CC graphs/s (one segmented device loop)", "value": value, "unit": "graphs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"er_batch_{args.graphs}", "graphs": args.graphs, "n": N, "m_directed": M,
                       "max_iterations": int(it_b.max()), "seed": 4,
                       "desc": "G(n,M) graphs, n log-uniform [100,200000], entries/vertex U(1.5,20)"},
            "gteps": M / (ms * 1e-3) / 1e9,
            "per_graph_plain_launches": {"graphs_per_s": total_graphs / plain_s, "seconds": plain_s},
            "speedup_vs_plain": (total_graphs / (ms * 1e-3)) / (total_graphs / plain_s),
            "identical_labels_and_iterations": same,
            "gpu_launches": int(launches), "clocks": clocks}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _warm_host_buffers(torch, pinned):
    """Copy every pinned trace buffer to the device once before the timed
    runs: the first device transfer out of a freshly pinned host buffer was
    measured at ~22 GB/s against ~210 GB/s for later ones, which would
    otherwise penalise whichever arm runs first.  Both arms then read the
    same, already transferred buffers (a server's long-lived staging
    buffers)."""
    biggest = max(max(rp.numel(), ci.numel()) for rp, ci, _ in pinned)
    dst = torch.empty(biggest, dtype=torch.int32, device="cuda")
    for rp, ci, _ in pinned:
        dst[:rp.numel()].copy_(rp, non_blocking=True)
        dst[:ci.numel()].copy_(ci, non_blocking=True)
    torch.cuda.synchronize()
    del dst


def run_serve(args, rank, world, local_rank):
    import torch

    import graphgen
    import paper_1910_05971_gb300 as fsv
    from paper_1910_05971_gb300.serve import Server

    if rank != 0:
        return  # the serving replay runs on one GPU; replicas would shard the trace
    torch.cuda.set_device(local_rank)
    R = args.requests
    tr = graphgen.trace(R, seed=5)
    t0 = time.time()
    # the trace lives in pinned host memory (generated before the replay), so
    # both arms copy to the device at full link speed
    pinned = []
    reqs = []
    for i in range(R):
        rp, ci = graphgen.trace_graph(tr, i)
        rp_h = torch.from_numpy(np.ascontiguousarray(rp, dtype=np.int32)).pin_memory()
        ci_h = torch.from_numpy(np.ascontiguousarray(ci if len(ci) else np.zeros(1, np.int32),
                                                     dtype=np.int32)).pin_memory()
        lab_h = torch.empty(max(len(rp) - 1, 1), dtype=torch.int32).pin_memory()
        pinned.append((rp_h, ci_h, lab_h))
        reqs.append((rp_h.numpy(), ci_h.numpy()[:len(ci)], lab_h.numpy()))
    m_tot = sum(len(c) for _, c, _ in reqs)
    _log(f"[bench] {R} requests, {m_tot} directed entries, generated in {time.time() - t0:.1f}s")
    arrivals = tr["t"] - tr["t"][0]

    # continuous batching
    srv = Server(hbm_budget_bytes=120 << 30, max_slots=1024, iters_per_step=2, k2_items=args.k2_items,
                 batch_sparse_div=args.batch_sparse_div)
    # warm-up: a few requests through the server
    for f in [srv.submit(reqs[i][0], reqs[i][1]) for i in range(min(4, R))]:
        f.result()
    srv.completed.clear()
    _warm_host_buffers(torch, pinned)
    launches0 = srv.backend.kernel_launches()
    futs = [None] * R
    start = time.perf_counter()

    def feeder():
        for i in range(R):
            dt = start + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            futs[i] = srv.submit(*reqs[i])  # rp, ci and a pinned label buffer
            futs[i].t_arrival = start + arrivals[i]

    th = threading.Thread(target=feeder)
    sampler = _clock_sampler(local_rank)
    sampler.start()
    th.start()
    th.join()
    results = [f.result() for f in futs]
    end = time.perf_counter()
    clocks = sampler.stop()
    lat = np.array([r.t_done - (start + arrivals[i]) for i, r in enumerate(
        sorted(srv.completed, key=lambda r: r.t_submit))])
    launches = srv.backend.kernel_launches() - launches0
    srv.close()
    gps = R / (end - start)

    # the same requests, one plain solve after another in arrival order
    solver = fsv.FastSV(rowptr_bits=32, k2_items=args.k2_items)
    solver.cc_host(pinned[0][0], pinned[0][1])
    base_lat = np.empty(R)
    same = True
    t_start = time.perf_counter()
    clock = 0.0
    # the plain arm writes into the same pinned label buffers: the served
    # results are copied out first
    served = [r[0].copy() for r in results]
    for i, (rp_h, ci_h, lab_h) in enumerate(pinned):
        begin = max(clock, arrivals[i])
        t = time.perf_counter()
        lab = solver.cc_host(rp_h, ci_h, lab_h)
        it = solver.stats()["iterations"]
        dur = time.perf_counter() - t
        clock = begin + dur
        base_lat[i] = clock - arrivals[i]
        n = len(reqs[i][0]) - 1
        same &= bool(np.array_equal(lab.numpy()[:n], served[i])) and it == results[i][1]
    base_gps = R / clock
    solver.close()
    print(json.dumps({
        "metric": "serve p50/p99 latency + graphs/s (continuous batching)", "value": gps, "unit": "graphs/s",
        "n_gpus": 1, "steps": R, "warmup": 4, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "config": {"workload": f"serve_trace_prefix_{R}", "requests": R, "m_directed_total": int(m_tot),
                   "rate_per_s": 2000, "hbm_budget_gb": 120, "iters_per_step": 2, "seed": 5,
                   "batch_sparse_div": args.batch_sparse_div},
        "per_graph_plain_launches": {"graphs_per_s": base_gps, "p50_ms": float(np.percentile(base_lat, 50) * 1e3),
                                     "p99_ms": float(np.percentile(base_lat, 99) * 1e3)},
        "identical_labels_and_iterations": bool(same), "gpu_launches": int(launches), "clocks": clocks}),
        flush=True)


def run_variants(args, rank, world, local_rank):
    """Iterations and device time of every solver variant on the same graph:
    the convergence ablation sv1..sv5 of Section 5.2 (Algorithm 1, then the
    optimizations of Sections 3.1-3.4 one at a time; sv5 is the default
    FastSV iteration) and the asynchronous mode.  Every variant must return
    the same labels.  One JSON line per workload."""
    import torch

    import graphgen
    import paper_1910_05971_gb300 as fsv

    if rank != 0:
        return  # one graph on one GPU; replicas would only repeat it
    torch.cuda.set_device(local_rank)
    names = args.variant_workloads.split(",")
    stream = torch.cuda.current_stream()
    for name in names:
        t0 = time.time()
        rp, ci = graphgen.WORKLOADS[name]()
        n, m = len(rp) - 1, len(ci)
        bits = 64 if m > np.iinfo(np.int32).max else 32
        rp_d = torch.from_numpy(rp.astype(np.int64 if bits == 64 else np.int32)).cuda()
        ci_d = torch.from_numpy(ci).cuda()
        del rp, ci
        _log(f"[bench] {name}: n={n} m={m} generated in {time.time() - t0:.1f}s")
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
        ref = None
        out = {}
        configs = [(f"sv{v}", dict(variant=v)) for v in (1, 2, 3, 4, 5)]
        configs.append(("async", dict(mode=fsv.FASTSV_MODE_ASYNC)))
        for key, kw in configs:
            s = fsv.FastSV(rowptr_bits=bits, max_iters=100000, **kw)
            s.cc(rp_d, ci_d, labels)  # untimed: first launches, workspace
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            its = []
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                s.cc(rp_d, ci_d, labels, check_status=False)
                its.append(s.stats()["iterations"])
            e1.record(stream)
            torch.cuda.synchronize()
            st = s.stats()
            s.close()
            ms = e0.elapsed_time(e1) / args.steps
            if ref is None:
                ref = labels.clone()
            same = bool(torch.equal(labels, ref))
            out[key] = {"iterations": its[-1], "iterations_all_steps": sorted(set(its)), "ms_per_solve": ms,
                        "gteps": m / (ms * 1e-3) / 1e9, "converged": bool(st["converged"]),
                        "labels_equal_sv1": same,
                        "loop": "device graph" if key in ("sv5", "async") else "host loop"}
        red = 1.0 - out["sv5"]["iterations"] / max(out["sv1"]["iterations"], 1)
        print(json.dumps({
            "metric": "iterations and time per solver variant (convergence ablation, Section 5.2)",
            "workload": name, "n": n, "m_directed": m, "steps": args.steps, "dtype": "int32",
            "data": "synthetic", "variants": out, "iteration_reduction_sv5_vs_sv1": red,
            "all_labels_equal": all(v["labels_equal_sv1"] for v in out.values()),
        }), flush=True)
        del rp_d, ci_d, labels, ref
        torch.cuda.empty_cache()

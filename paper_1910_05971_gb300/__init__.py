"""FastSV connected components on one GB300 GPU.

Zhang, Azad, Hu, "FastSV: A Distributed-Memory Connected Component Algorithm
with Fast Convergence" (arXiv:1910.05971): Algorithm 2 run on the device by
hand-written sm_103a CUDA kernels behind the C ABI of include/fastsv.h.

    import torch, paper_1910_05971_gb300 as fsv
    with fsv.FastSV() as solver:
        labels = solver.cc(row_ptr, col_idx)      # CUDA tensors (int64/int32)
        print(solver.stats()["iterations"])

labels[u] is the smallest vertex id of u's connected component.  PyTorch is
used only for device memory and streams; the arithmetic runs in libfastsv.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _lib
from ._lib import (  # noqa: F401  (re-exported C names)
    FASTSV_OK, FASTSV_ERR_INVALID_ARG, FASTSV_ERR_OOM, FASTSV_ERR_CUDA, FASTSV_ERR_MAX_ITERS,
    FASTSV_ERR_TIMEOUT, FASTSV_ERR_UNSUPPORTED, FASTSV_ERR_INVALID_GRAPH, FASTSV_ERR_FULL,
    FASTSV_MODE_SYNC, FASTSV_MODE_ASYNC, FastSVError, fastsv_options, fastsv_stats,
    fastsv_default_options, fastsv_create, fastsv_destroy, fastsv_cc, fastsv_cc_host, fastsv_cc_batched,
    fastsv_get_stats, fastsv_status_string, fastsv_last_cuda_error, fastsv_kernel_launches,
    fastsv_pool_create, fastsv_pool_bytes, fastsv_pool_add, fastsv_pool_step, fastsv_pool_poll,
    fastsv_pool_usage, load, library_path, fastsv_cc_noalloc, FASTSV_NOALLOC_MAX_VERTICES,
    fastsv_pool_checkpoint_bytes, fastsv_pool_evict, fastsv_pool_restore, fastsv_pool_step_times,
    fastsv_tune_key, TUNE_SINGLE, TUNE_BATCHED,
)

# the tuning cache the autotuner (tune.py) wrote on GB300 for the shape
# classes of the standard workloads; handles use it unless told otherwise
DEFAULT_TUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.txt")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("FastSV needs a CUDA device; none is available")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def stats_dict(s: fastsv_stats) -> dict:
    return dict(n=s.n, m=s.m, iterations=s.iterations, status=s.status, converged=bool(s.converged),
                ms_total=s.ms_total, ms_setup=s.ms_setup, ms_k2=s.ms_k2, ms_k3=s.ms_k3, ms_push=s.ms_push,
                ms_hook=s.ms_hook, sparse_iters=s.sparse_iters, dense_iters=s.dense_iters,
                col_blocks=s.col_blocks, changed_per_iter=[int(s.changed_per_iter[i]) for i in range(s.trace_len)],
                timed_iters=s.timed_iters, timed_dense_iters=s.timed_dense_iters, tuned=bool(s.tuned),
                block_runs=s.block_runs)


class FastSV:
    """One library handle (one workspace).  Not thread-safe.

    The kernel choices k2_items, k2_threads, col_blocks, sparse_div and
    batch_sparse_div default to None: the library's defaults, or, for a
    graph whose shape class has an entry in the tuning cache, the tuned
    values.  ``tune_cache``: path of a tuning cache ("default": the packaged
    cache, if present; None: none).  Passing any of the five kernel choices
    explicitly turns the default cache off, so that the values given are the
    values used."""

    def __init__(self, rowptr_bits: int = 64, mode: int = FASTSV_MODE_SYNC, max_iters: int = 4096,
                 validate: int = 0, use_graph: bool = True, k2_items: int | None = None, grid_ctas_per_sm: int = 0,
                 timing: bool = True, fail_alloc_after: int = 0, col_blocks: int | None = None,
                 k2_threads: int | None = None, sparse_div: int | None = None, variant: int = 0,
                 batch_sparse_div: int | None = None, col_block_mib: int = 64, pool_wait_copies: bool = False,
                 tune_cache: str | None = "default"):
        _torch()
        o = fastsv_default_options()
        o.rowptr_bits = rowptr_bits
        o.mode = mode
        o.max_iters = max_iters
        o.validate = validate
        o.use_graph = int(use_graph)
        o.grid_ctas_per_sm = grid_ctas_per_sm
        o.timing = int(timing)
        o.fail_alloc_after = fail_alloc_after
        o.variant = variant
        o.col_block_mib = col_block_mib
        o.pool_wait_copies = int(pool_wait_copies)
        chosen = dict(k2_items=k2_items, k2_threads=k2_threads, col_blocks=col_blocks, sparse_div=sparse_div,
                      batch_sparse_div=batch_sparse_div)
        for name, value in chosen.items():
            if value is not None:
                setattr(o, name, value)
        if tune_cache == "default":
            explicit = any(v is not None for v in chosen.values())
            tune_cache = DEFAULT_TUNE_CACHE if (os.path.exists(DEFAULT_TUNE_CACHE) and not explicit) else None
        self._tune_path = tune_cache.encode() if tune_cache else None  # kept alive for the call below
        o.tune_cache = self._tune_path
        self.options = o
        self.h = fastsv_create(o)

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            fastsv_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- solves -----------------------------------------------------------
    def cc(self, row_ptr, col_idx, labels=None, stream=None, check_status: bool = True):
        """Labels of one graph.  row_ptr: CUDA int64 (or int32 with
        rowptr_bits=32) tensor of n+1 entries; col_idx: CUDA int32 tensor."""
        torch = _torch()
        n = row_ptr.numel() - 1
        want = torch.int64 if self.options.rowptr_bits == 64 else torch.int32
        assert row_ptr.dtype == want and row_ptr.is_cuda and row_ptr.is_contiguous()
        assert col_idx.dtype == torch.int32 and col_idx.is_cuda and col_idx.is_contiguous()
        if labels is None:
            labels = torch.empty(max(n, 0), dtype=torch.int32, device=row_ptr.device)
        st = fastsv_cc(self.h, n, row_ptr.data_ptr(), col_idx.data_ptr() if col_idx.numel() else None,
                       labels.data_ptr() if n > 0 else None, _stream_ptr(stream))
        _lib.check(st, "fastsv_cc")
        if check_status:
            self.check_last()
        return labels

    def cc_host(self, row_ptr, col_idx, labels=None, stream=None):
        """Labels of one graph from host (CPU, preferably pinned) tensors; the
        host-to-device copies and the copy back are part of the call."""
        torch = _torch()
        n = row_ptr.numel() - 1
        assert not row_ptr.is_cuda and not col_idx.is_cuda
        if labels is None:
            labels = torch.empty(max(n, 0), dtype=torch.int32, pin_memory=True)
        st = fastsv_cc_host(self.h, n, row_ptr.data_ptr(), col_idx.data_ptr() if col_idx.numel() else None,
                            labels.data_ptr() if n > 0 else None, _stream_ptr(stream))
        _lib.check(st, "fastsv_cc_host")
        return labels

    def cc_batched(self, vtx_off, edge_off, row_ptr, col_idx, labels=None, iters=None, stream=None,
                   check_status: bool = True):
        """Labels (local ids) and per-graph iteration counts of a batch of
        independent graphs in concatenated CSR form (CUDA tensors)."""
        torch = _torch()
        G = vtx_off.numel() - 1
        N = int(vtx_off[-1].item()) if G > 0 else 0
        dev = vtx_off.device
        if labels is None:
            labels = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
        if iters is None:
            iters = torch.zeros(max(G, 1), dtype=torch.int32, device=dev)
        st = fastsv_cc_batched(self.h, G, vtx_off.data_ptr(), edge_off.data_ptr(), row_ptr.data_ptr(),
                               col_idx.data_ptr() if col_idx.numel() else None, labels.data_ptr(),
                               iters.data_ptr(), _stream_ptr(stream))
        _lib.check(st, "fastsv_cc_batched")
        if check_status:
            self.check_last()
        return labels[:N], iters[:G]

    # -- results ----------------------------------------------------------
    def stats_raw(self) -> tuple[int, fastsv_stats]:
        return fastsv_get_stats(self.h)

    def stats(self) -> dict:
        st, s = fastsv_get_stats(self.h)
        d = stats_dict(s)
        d["status"] = st
        return d

    def check_last(self):
        st, _ = fastsv_get_stats(self.h)
        _lib.check(st, "solve")

    def kernel_launches(self) -> int:
        return fastsv_kernel_launches(self.h)


def cc(row_ptr, col_idx, **kw):
    """One-shot convenience: labels of one graph (CUDA tensors)."""
    bits = 64 if str(row_ptr.dtype).endswith("int64") else 32
    with FastSV(rowptr_bits=bits, **kw) as s:
        lab = s.cc(row_ptr, col_idx)
        return lab, s.stats()

"""Thin ctypes binding of libfastsv (include/fastsv.h).

The functions below carry the C names and only marshal arguments: every step
of a solve runs in the library's CUDA kernels.  There is no fallback: if the
compiled library is missing or no CUDA device is present the calls raise.
PyTorch is used only for device memory and the current stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

FASTSV_OK = 0
FASTSV_ERR_INVALID_ARG = 1
FASTSV_ERR_OOM = 2
FASTSV_ERR_CUDA = 3
FASTSV_ERR_MAX_ITERS = 4
FASTSV_ERR_TIMEOUT = 5
FASTSV_ERR_UNSUPPORTED = 6
FASTSV_ERR_INVALID_GRAPH = 7
FASTSV_ERR_FULL = 8

FASTSV_MODE_SYNC = 0
FASTSV_MODE_ASYNC = 1

STATUS_NAMES = {
    0: "FASTSV_OK", 1: "FASTSV_ERR_INVALID_ARG", 2: "FASTSV_ERR_OOM", 3: "FASTSV_ERR_CUDA",
    4: "FASTSV_ERR_MAX_ITERS", 5: "FASTSV_ERR_TIMEOUT", 6: "FASTSV_ERR_UNSUPPORTED",
    7: "FASTSV_ERR_INVALID_GRAPH", 8: "FASTSV_ERR_FULL",
}


class fastsv_options(C.Structure):
    _fields_ = [
        ("rowptr_bits", C.c_int32),
        ("mode", C.c_int32),
        ("max_iters", C.c_int32),
        ("validate", C.c_int32),
        ("use_graph", C.c_int32),
        ("k2_items", C.c_int32),
        ("grid_ctas_per_sm", C.c_int32),
        ("timing", C.c_int32),
        ("fail_alloc_after", C.c_int32),
        ("col_blocks", C.c_int32),
        ("k2_threads", C.c_int32),
        ("sparse_div", C.c_int32),
        ("variant", C.c_int32),
        ("batch_sparse_div", C.c_int32),
        ("col_block_mib", C.c_int32),
        ("pool_wait_copies", C.c_int32),
        ("tune_cache", C.c_char_p),
    ]


class fastsv_stats(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("m", C.c_int64),
        ("iterations", C.c_int64),
        ("status", C.c_int32),
        ("converged", C.c_int32),
        ("ms_total", C.c_float),
        ("ms_setup", C.c_float),
        ("ms_k2", C.c_float),
        ("ms_k3", C.c_float),
        ("ms_push", C.c_float),
        ("ms_hook", C.c_float),
        ("sparse_iters", C.c_int32),
        ("dense_iters", C.c_int32),
        ("trace_len", C.c_int32),
        ("col_blocks", C.c_int32),
        ("changed_per_iter", C.c_int64 * 64),
        ("timed_iters", C.c_int32),
        ("timed_dense_iters", C.c_int32),
        ("tuned", C.c_int32),
        ("pad0", C.c_int32),
        ("block_runs", C.c_int64),
    ]


class FastSVError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) for every entry point of include/fastsv.h
_P = C.c_void_p
_SIGNATURES = [
    ("fastsv_default_options", None, [C.POINTER(fastsv_options)]),
    ("fastsv_create", C.c_int, [C.POINTER(_P), C.POINTER(fastsv_options)]),
    ("fastsv_destroy", C.c_int, [_P]),
    ("fastsv_cc", C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    ("fastsv_cc_host", C.c_int, [_P, C.c_int64, _P, _P, _P, _P]),
    ("fastsv_cc_batched", C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P, _P, _P]),
    ("fastsv_get_stats", C.c_int, [_P, C.POINTER(fastsv_stats)]),
    ("fastsv_status_string", C.c_char_p, [C.c_int]),
    ("fastsv_last_cuda_error", C.c_int32, [_P]),
    ("fastsv_kernel_launches", C.c_int64, [_P]),
    ("fastsv_pool_create", C.c_int, [_P, C.c_size_t, C.c_int32]),
    ("fastsv_pool_bytes", C.c_size_t, [C.c_int64, C.c_int64]),
    ("fastsv_pool_add", C.c_int, [_P, C.c_int64, _P, _P, _P, C.POINTER(C.c_int32)]),
    ("fastsv_pool_step", C.c_int, [_P, C.c_int32, _P]),
    ("fastsv_pool_poll", C.c_int, [_P, _P, _P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("fastsv_pool_usage", C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_size_t)]),
    ("fastsv_pool_step_times", C.c_int, [_P, _P]),
    ("fastsv_pool_checkpoint_bytes", C.c_size_t, [C.c_int64]),
    ("fastsv_pool_evict", C.c_int, [_P, C.c_int32, _P]),
    ("fastsv_pool_restore", C.c_int, [_P, C.c_int64, _P, _P, _P, _P, C.POINTER(C.c_int32)]),
    ("fastsv_cc_noalloc", C.c_int, [C.c_int64, _P, _P, _P, C.c_int32, C.POINTER(C.c_int32), _P]),
    ("fastsv_tune_key", C.c_int32, [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_char_p, C.c_int32]),
]

# largest vertex count of fastsv_cc_noalloc (FASTSV_NOALLOC_MAX_VERTICES)
FASTSV_NOALLOC_MAX_VERTICES = 1 << 20


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load the compiled library (building it first if needed).  Raises if
    it cannot be built or loaded: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libfastsv.so not found at {path}; run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, res, args in _SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _call(name: str, *args) -> int:
    return getattr(load(), name)(*args)


def check(status: int, where: str, allow=(FASTSV_OK,)) -> int:
    if status not in allow:
        raise FastSVError(status, where)
    return status


# ---------------------------------------------------------------------------
# the C entry points, same names, argument marshalling only
# ---------------------------------------------------------------------------

def fastsv_default_options() -> fastsv_options:
    o = fastsv_options()
    _call("fastsv_default_options", C.byref(o))
    return o


def fastsv_create(opt: fastsv_options | None = None) -> int:
    h = C.c_void_p()
    st = _call("fastsv_create", C.byref(h), C.byref(opt) if opt is not None else None)
    check(st, "fastsv_create")
    return h.value


def fastsv_destroy(h: int) -> int:
    return _call("fastsv_destroy", h)


def fastsv_cc(h: int, n: int, row_ptr: int, col_idx: int, labels_out: int, stream: int) -> int:
    return _call("fastsv_cc", h, n, row_ptr, col_idx, labels_out, stream)


def fastsv_cc_host(h: int, n: int, row_ptr_host: int, col_idx_host: int, labels_host: int, stream: int) -> int:
    return _call("fastsv_cc_host", h, n, row_ptr_host, col_idx_host, labels_host, stream)


def fastsv_cc_batched(h: int, num_graphs: int, vtx_off: int, edge_off: int, row_ptr: int, col_idx: int,
                      labels_out: int, iters_out: int | None, stream: int) -> int:
    return _call("fastsv_cc_batched", h, num_graphs, vtx_off, edge_off, row_ptr, col_idx, labels_out, iters_out,
                 stream)


def fastsv_get_stats(h: int) -> tuple[int, fastsv_stats]:
    s = fastsv_stats()
    st = _call("fastsv_get_stats", h, C.byref(s))
    return st, s


def fastsv_status_string(status: int) -> str:
    return _call("fastsv_status_string", status).decode()


def fastsv_last_cuda_error(h: int) -> int:
    return _call("fastsv_last_cuda_error", h)


def fastsv_kernel_launches(h: int) -> int:
    return _call("fastsv_kernel_launches", h)


def fastsv_pool_create(h: int, hbm_budget_bytes: int, max_slots: int) -> int:
    return _call("fastsv_pool_create", h, hbm_budget_bytes, max_slots)


def fastsv_pool_bytes(n: int, m: int) -> int:
    return _call("fastsv_pool_bytes", n, m)


def fastsv_pool_add(h: int, n: int, row_ptr_host: int, col_idx_host: int, labels_host: int) -> tuple[int, int]:
    slot = C.c_int32(-1)
    st = _call("fastsv_pool_add", h, n, row_ptr_host, col_idx_host, labels_host, C.byref(slot))
    return st, slot.value


def fastsv_pool_step(h: int, iters: int, stream: int) -> int:
    return _call("fastsv_pool_step", h, iters, stream)


def fastsv_pool_poll(h: int, done_slots: int, done_iters: int | None, cap: int) -> tuple[int, int, int]:
    n_done = C.c_int32(0)
    n_active = C.c_int32(0)
    st = _call("fastsv_pool_poll", h, done_slots, done_iters, cap, C.byref(n_done), C.byref(n_active))
    return st, n_done.value, n_active.value


def fastsv_pool_usage(h: int) -> tuple[int, int, int]:
    used = C.c_int32(0)
    b = C.c_size_t(0)
    st = _call("fastsv_pool_usage", h, C.byref(used), C.byref(b))
    return st, used.value, b.value


def fastsv_pool_step_times(h: int) -> tuple[int, list[float]]:
    """(status, [ms waiting for admission copies, ms admit + rebuild, ms iterations]) of the last step."""
    out = (C.c_float * 3)()
    st = _call("fastsv_pool_step_times", h, C.cast(out, C.c_void_p))
    return st, [out[0], out[1], out[2]]


def fastsv_pool_checkpoint_bytes(n: int) -> int:
    return _call("fastsv_pool_checkpoint_bytes", n)


def fastsv_pool_evict(h: int, slot: int, checkpoint_host: int) -> int:
    return _call("fastsv_pool_evict", h, slot, checkpoint_host)


def fastsv_pool_restore(h: int, n: int, row_ptr_host: int, col_idx_host: int | None, labels_host: int | None,
                        checkpoint_host: int) -> tuple[int, int]:
    slot = C.c_int32(-1)
    st = _call("fastsv_pool_restore", h, n, row_ptr_host, col_idx_host, labels_host, checkpoint_host,
               C.byref(slot))
    return st, slot.value


def fastsv_cc_noalloc(n: int, row_ptr: int, col_idx: int | None, labels_out: int, max_iters: int,
                      stream: int) -> tuple[int, int]:
    """Allocation-free solve (see include/fastsv.h): returns (status, iterations)."""
    it = C.c_int32(0)
    st = _call("fastsv_cc_noalloc", n, row_ptr, col_idx, labels_out, max_iters, C.byref(it), stream)
    return st, it.value


TUNE_SINGLE = 0
TUNE_BATCHED = 1


def fastsv_tune_key(kind: int, n: int, m: int, graphs: int = 1, rowptr_bits: int = 64) -> str:
    """Shape-class key of the tuning cache (see include/fastsv.h)."""
    buf = C.create_string_buffer(128)
    k = _call("fastsv_tune_key", kind, n, m, graphs, rowptr_bits, buf, 128)
    if k < 0:
        raise ValueError("fastsv_tune_key: bad argument")
    return buf.value.decode()

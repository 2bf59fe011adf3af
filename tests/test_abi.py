"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares (host-only checks; no kernel runs without a GPU)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*[A-Za-z_][\w \*]*?\b(fastsv_\w+)\s*\(", src, re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import paper_1910_05971_gb300 as fsv
    lib = fsv.load()
    names = _declared()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1910_05971_gb300 as fsv
    for n in _declared():
        assert hasattr(fsv, n), f"binding lacks {n}"


def test_host_only_entry_points():
    import paper_1910_05971_gb300 as fsv
    o = fsv.fastsv_default_options()
    assert (o.rowptr_bits, o.mode, o.max_iters, o.use_graph, o.k2_items) == (64, 0, 4096, 1, 8)
    assert C.sizeof(fsv.fastsv_options) == 72
    assert C.sizeof(fsv.fastsv_stats) == 608
    assert fsv.fastsv_status_string(fsv.FASTSV_ERR_MAX_ITERS) == "FASTSV_ERR_MAX_ITERS"
    assert fsv.fastsv_pool_bytes(10, 20) > 0
    # invalid handles are rejected on the host without touching a device
    assert fsv._lib.load().fastsv_destroy(None) == fsv.FASTSV_ERR_INVALID_ARG
    assert fsv._lib.load().fastsv_cc(None, 5, None, None, None, None) == fsv.FASTSV_ERR_INVALID_ARG
    assert o.variant == 0 and o.sparse_div == 2 and o.k2_threads == 256 and o.batch_sparse_div == 0


def test_option_validation_is_host_only():
    """Bad options are refused by fastsv_create before any CUDA call."""
    import paper_1910_05971_gb300 as fsv
    lib = fsv._lib.load()
    for field, value in (("variant", 6), ("variant", -1), ("mode", 2), ("rowptr_bits", 16), ("max_iters", 0),
                         ("sparse_div", -1), ("batch_sparse_div", -3)):
        o = fsv.fastsv_default_options()
        setattr(o, field, value)
        h = C.c_void_p()
        assert lib.fastsv_create(C.byref(h), C.byref(o)) == fsv.FASTSV_ERR_INVALID_ARG, field
        assert not h.value
    o = fsv.fastsv_default_options()
    o.mode = fsv.FASTSV_MODE_ASYNC
    o.variant = 3  # the ablation is defined for the synchronous iteration only
    h = C.c_void_p()
    assert lib.fastsv_create(C.byref(h), C.byref(o)) == fsv.FASTSV_ERR_INVALID_ARG


def test_library_is_built_for_sm_103a_only():
    from paper_1910_05971_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(_build.LIB)

"""CPU oracle for FastSV connected components -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, compiled with gcc):

* ``fastsv(..., form="alg2")``  Algorithm 2 of the paper (Section 3), edge form,
  f / f_next separation, early termination on an unchanged f[f] (Section 3.4).
* ``fastsv(..., form="alg3")``  Algorithm 3 (Section 4.1), the GraphBLAS form.
* ``fastsv(..., form="omp")``   Algorithm 2 with OpenMP loops and atomic min;
  identical per iteration to the sequential form.
* ``fastsv(..., form="sv1".."sv5")``  the convergence ablation of Section 5.2:
  Algorithm 1 (Section 2.4), then grandparent hooking (3.1), stochastic hooking
  (3.2), aggressive hooking with Algorithm 2's single-pass body (3.3) and early
  termination (3.4) added one at a time; sv5 is Algorithm 2.
* ``uf`` / ``bfs``  the exact result: every vertex labelled with the smallest
  vertex id of its connected component (the converged state, Section 3.4).

Pins (tests/test_oracle.py): hand-derived per-iteration traces of Algorithm 2
(tests/golden/), exhaustive agreement with BFS on every graph of at most five
vertices, closed forms (paths, stars, cliques, isolated vertices, full and
empty lattices), Lemma 1 of Appendix A, the early-termination theorem, the
Algorithm 2 / Algorithm 3 equivalence, and planted mistakes (MUTANT builds)
that each of those pins catches.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_libs: dict[int, C.CDLL] = {}
_lock = threading.Lock()


def _so_path(mutant: int) -> str:
    return os.path.join(_BUILD, "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, OpenMP); ``mutant`` > 0 plants a mistake."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _so_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", f"-DMUTANT={mutant}", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load(mutant: int = 0) -> C.CDLL:
    with _lock:
        if mutant in _libs:
            return _libs[mutant]
        lib = C.CDLL(build(mutant))
        i64, p, i32 = C.c_int64, C.c_void_p, C.c_int
        for name in ("oracle_fastsv_alg2", "oracle_fastsv_alg3"):
            fn = getattr(lib, name)
            fn.argtypes = [i64, p, p, p, i64, p, i64, p]
            fn.restype = i64
        lib.oracle_fastsv_sv.argtypes = [i64, p, p, p, i32, i64, p, i64, p]
        lib.oracle_fastsv_sv.restype = i64
        lib.oracle_sv_iteration.argtypes = [i64, p, p, p, p, p, i32]
        lib.oracle_sv_iteration.restype = i64
        lib.oracle_fastsv_omp.argtypes = [i64, p, p, p, i64, p, i64, p, i32]
        lib.oracle_fastsv_omp.restype = i64
        lib.oracle_alg2_iteration.argtypes = [i64, p, p, p, p, p]
        lib.oracle_alg2_iteration.restype = i64
        lib.oracle_uf.argtypes = [i64, p, p, p]
        lib.oracle_uf.restype = None
        lib.oracle_bfs.argtypes = [i64, p, p, p]
        lib.oracle_bfs.restype = None
        _libs[mutant] = lib
        return lib


def _csr(rp, ci):
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    n = len(rp) - 1
    assert n >= 0 and rp[0] == 0 and rp[-1] == len(ci)
    return n, rp, ci


def fastsv(rp, ci, max_iters: int = 0, form: str = "alg2", nthreads: int = 0, trace_cap: int = 4096,
           mutant: int = 0):
    """Run FastSV on a CSR graph.

    Returns ``(f, iterations, converged, changed)``: the parent vector after the
    last iteration (equal to the labels on convergence), the number of
    iterations executed, whether the last one found f[f] unchanged, and the
    per-iteration count of changed grandparents.  ``max_iters`` <= 0 runs to
    convergence.  ``form="sv1"`` .. ``"sv5"`` runs the convergence ablation of
    Section 5.2 (Algorithm 1 plus the optimizations of Sections 3.1-3.4 one at a
    time; sv5 is Algorithm 2); for sv1..sv4 the trace counts changed f.
    """
    n, rp, ci = _csr(rp, ci)
    lib = _load(mutant)
    f = np.empty(max(n, 1), dtype=np.int32)
    trace = np.zeros(trace_cap, dtype=np.int64)
    conv = np.zeros(1, dtype=np.int32)
    args = [n, rp.ctypes.data, ci.ctypes.data, f.ctypes.data, max_iters, trace.ctypes.data, trace_cap,
            conv.ctypes.data]
    if form == "alg2":
        it = lib.oracle_fastsv_alg2(*args)
    elif form == "alg3":
        it = lib.oracle_fastsv_alg3(*args)
    elif form == "omp":
        it = lib.oracle_fastsv_omp(*args, nthreads)
    elif form in ("sv1", "sv2", "sv3", "sv4", "sv5"):
        it = lib.oracle_fastsv_sv(n, rp.ctypes.data, ci.ctypes.data, f.ctypes.data, int(form[2]), max_iters,
                                  trace.ctypes.data, trace_cap, conv.ctypes.data)
    else:
        raise ValueError(form)
    return f[:n], int(it), bool(conv[0]), trace[:min(it, trace_cap)].copy()


def iteration(rp, ci, f, mutant: int = 0) -> int:
    """Apply one Algorithm 2 iteration to ``f`` in place; return the number of
    grandparents f[f] that changed."""
    n, rp, ci = _csr(rp, ci)
    assert f.dtype == np.int32 and f.flags.c_contiguous and len(f) == n
    if n == 0:
        return 0
    fn = np.empty(n, dtype=np.int32)
    gp = np.empty(n, dtype=np.int32)
    return int(_load(mutant).oracle_alg2_iteration(n, rp.ctypes.data, ci.ctypes.data, f.ctypes.data,
                                                   fn.ctypes.data, gp.ctypes.data))


def sv_iteration(rp, ci, f, variant: int, mutant: int = 0) -> int:
    """Apply one iteration of ablation variant sv1..sv4 to ``f`` in place;
    return the number of entries of f that changed."""
    n, rp, ci = _csr(rp, ci)
    assert f.dtype == np.int32 and f.flags.c_contiguous and len(f) == n and 1 <= variant <= 4
    if n == 0:
        return 0
    fn = np.empty(n, dtype=np.int32)
    fs = np.empty(n, dtype=np.int32)
    return int(_load(mutant).oracle_sv_iteration(n, rp.ctypes.data, ci.ctypes.data, f.ctypes.data,
                                                 fn.ctypes.data, fs.ctypes.data, variant))


def uf(rp, ci) -> np.ndarray:
    """Smallest vertex id of each vertex's component (union-find)."""
    n, rp, ci = _csr(rp, ci)
    out = np.empty(max(n, 1), dtype=np.int32)
    _load().oracle_uf(n, rp.ctypes.data, ci.ctypes.data, out.ctypes.data)
    return out[:n]


def bfs(rp, ci) -> np.ndarray:
    """Smallest vertex id of each vertex's component (breadth-first search)."""
    n, rp, ci = _csr(rp, ci)
    out = np.empty(max(n, 1), dtype=np.int32)
    _load().oracle_bfs(n, rp.ctypes.data, ci.ctypes.data, out.ctypes.data)
    return out[:n]


def csr_from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric CSR (both directions, rows sorted, duplicates kept) from an
    undirected edge list.  Small test graphs only."""
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
        if u != v:
            rows[v].append(u)
    rp = np.zeros(n + 1, dtype=np.int64)
    for u in range(n):
        rp[u + 1] = rp[u] + len(rows[u])
    ci = np.array([v for r in rows for v in sorted(r)], dtype=np.int32)
    return rp, ci

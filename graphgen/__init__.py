"""Seeded synthetic graph generators shared by the oracle and the CUDA path.

This module is input plumbing only: it draws edges from a counter-based
SplitMix64 generator and builds symmetric CSR arrays (self-loops and duplicate
entries removed, rows sorted).  It contains none of the connected-components
arithmetic, so both sides of every parity test can take their inputs from it.

The workload recipes below stand in for the real graphs of the FastSV paper
(Section 5, Table 1: web crawls, protein k-mer graphs, social networks), which
are not available offline:

* ``rmat_s16``  - R-MAT scale 16, edge factor 16, a/b/c/d = .57/.19/.19/.05, seed 1.
* ``grid``      - 4096 x 4096 lattice, each edge kept with p = 0.55, plus 10^6
                  isolated vertices appended, seed 2 (high diameter, many components).
* ``rmat_s26``  - R-MAT scale 26, edge factor 16, vertex ids relabelled by a
                  Fisher-Yates permutation (seed 3), int64 row_ptr.
* ``er_batch``  - 4096 Erdos-Renyi G(n, M) graphs, n log-uniform in [100, 200000],
                  directed entries per vertex uniform in [1.5, 20], seed 4.
* ``trace``     - serving requests: Poisson arrivals at 2000/s, undirected edge
                  target log-uniform in [1e3, 5e7], half R-MAT, half lattice, seed 5.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgraphgen.so")
_lib = None
_lock = threading.Lock()

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile graphgen.c with gcc (OpenMP, no FMA contraction) into _build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        i64, u64, i32, f64, p = C.c_int64, C.c_uint64, C.c_int, C.c_double, C.c_void_p
        lib.graphgen_rmat_degrees.argtypes = [i32, i64, f64, f64, f64, u64, p, p]
        lib.graphgen_rmat_degrees.restype = i64
        lib.graphgen_rmat_fill.argtypes = [i32, i64, f64, f64, f64, u64, p, p, p, p, p]
        lib.graphgen_rmat_fill.restype = i64
        lib.graphgen_permutation.argtypes = [i64, u64, p]
        lib.graphgen_permutation.restype = None
        lib.graphgen_grid.argtypes = [i64, i64, f64, u64, p, p]
        lib.graphgen_grid.restype = i64
        lib.graphgen_er_params.argtypes = [i64, u64, f64, f64, f64, f64, p, p]
        lib.graphgen_er_params.restype = None
        lib.graphgen_er_fill.argtypes = [i64, u64, p, p, p, p, p]
        lib.graphgen_er_fill.restype = None
        lib.graphgen_er_pack.argtypes = [i64, p, p, p, p]
        lib.graphgen_er_pack.restype = None
        lib.graphgen_trace.argtypes = [i64, u64, f64, f64, f64, p, p, p, p, p, p]
        lib.graphgen_trace.restype = None
        lib.graphgen_word.argtypes = [u64, u64, u64]
        lib.graphgen_word.restype = u64
        lib.graphgen_exp.argtypes = [f64]
        lib.graphgen_exp.restype = f64
        lib.graphgen_log.argtypes = [f64]
        lib.graphgen_log.restype = f64
        _lib = lib
        return lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def word(seed: int, stream: int, idx: int) -> int:
    return int(_load().graphgen_word(seed, stream, idx))


def permutation(n: int, seed: int) -> np.ndarray:
    perm = np.empty(n, dtype=np.int32)
    _load().graphgen_permutation(n, seed, _ptr(perm))
    return perm


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, abc=RMAT_ABC, permute: bool = False,
         perm_seed: int | None = None):
    """R-MAT graph on 2^scale vertices from edge_factor * 2^scale draws.

    Returns (row_ptr int64[n+1], col_idx int32[m]), symmetric, sorted rows,
    no self-loops or duplicates.  With ``permute`` the vertex ids are relabelled
    by a Fisher-Yates permutation (seed ``perm_seed``, default ``seed``) before
    duplicates are removed.
    """
    lib = _load()
    n = 1 << scale
    draws = edge_factor * n
    a, b, c = abc
    perm = permutation(n, perm_seed if perm_seed is not None else seed) if permute else None
    deg = np.zeros(n, dtype=np.int64)
    raw = lib.graphgen_rmat_degrees(scale, draws, a, b, c, seed, _ptr(perm), _ptr(deg))
    rp_raw = np.empty(n + 1, dtype=np.int64)
    rp_raw[0] = 0
    np.cumsum(deg, out=rp_raw[1:])
    assert rp_raw[n] == raw
    col = np.empty(max(raw, 1), dtype=np.int32)
    rp = np.empty(n + 1, dtype=np.int64)
    m = lib.graphgen_rmat_fill(scale, draws, a, b, c, seed, _ptr(perm), _ptr(rp_raw), _ptr(deg), _ptr(col), _ptr(rp))
    del deg, rp_raw, perm
    if m < raw // 2:
        col = col[:m].copy()
    else:
        col = col[:m]
    return rp, col


def grid(side: int, p: float, extra: int = 0, seed: int = 2):
    """side x side lattice (id = r*side + c), each right/down edge kept with
    probability p, plus ``extra`` isolated vertices.  Returns (rp int64, ci int32)."""
    lib = _load()
    n = side * side + extra
    rp = np.empty(n + 1, dtype=np.int64)
    m = lib.graphgen_grid(side, extra, p, seed, _ptr(rp), None)
    col = np.empty(max(m, 1), dtype=np.int32)
    lib.graphgen_grid(side, extra, p, seed, _ptr(rp), _ptr(col))
    return rp, col[:m]


class Batch:
    """A batch of independent CSR graphs in concatenated form.

    vtx_off  int64[G+1]  graph g owns batch vertices [vtx_off[g], vtx_off[g+1])
    edge_off int64[G+1]  graph g's entries are col_idx[edge_off[g] : edge_off[g+1]]
    row_ptr  int32[sum(n_g + 1)]  graph g's LOCAL row_ptr (starts at 0, ends at m_g)
                          occupies row_ptr[vtx_off[g] + g : vtx_off[g+1] + g + 1]
    col_idx  int32[sum m_g]  LOCAL neighbour ids of graph g
    """

    def __init__(self, vtx_off, edge_off, row_ptr, col_idx):
        self.vtx_off = vtx_off
        self.edge_off = edge_off
        self.row_ptr = row_ptr
        self.col_idx = col_idx

    @property
    def num_graphs(self) -> int:
        return len(self.vtx_off) - 1

    def graph(self, g: int):
        """Graph g as a standalone (rp int64, ci int32) CSR with local ids."""
        v0, v1 = int(self.vtx_off[g]), int(self.vtx_off[g + 1])
        e0, e1 = int(self.edge_off[g]), int(self.edge_off[g + 1])
        rp = self.row_ptr[v0 + g: v1 + g + 1].astype(np.int64)
        return rp, self.col_idx[e0:e1]

    @staticmethod
    def from_graphs(graphs):
        """Concatenate a list of (rp, ci) CSR graphs."""
        G = len(graphs)
        vtx_off = np.zeros(G + 1, dtype=np.int64)
        edge_off = np.zeros(G + 1, dtype=np.int64)
        for g, (rp, ci) in enumerate(graphs):
            vtx_off[g + 1] = vtx_off[g] + (len(rp) - 1)
            edge_off[g + 1] = edge_off[g] + len(ci)
        row_ptr = np.concatenate([np.asarray(rp, dtype=np.int32) for rp, _ in graphs]) if G else np.zeros(0, np.int32)
        col_idx = (np.concatenate([np.asarray(ci, dtype=np.int32) for _, ci in graphs]) if G
                   else np.zeros(0, np.int32))
        return Batch(vtx_off, edge_off, row_ptr, col_idx)


def er_params(G: int, seed: int = 4, nmin: float = 100, nmax: float = 200000, dmin: float = 1.5, dmax: float = 20):
    n_g = np.empty(G, dtype=np.int64)
    draws = np.empty(G, dtype=np.int64)
    _load().graphgen_er_params(G, seed, nmin, nmax, dmin, dmax, _ptr(n_g), _ptr(draws))
    return n_g, draws


def er_batch(G: int = 4096, seed: int = 4, nmin: float = 100, nmax: float = 200000, dmin: float = 1.5,
             dmax: float = 20) -> Batch:
    """G Erdos-Renyi G(n, M) graphs: n_g log-uniform in [nmin, nmax], directed
    entries per vertex uniform in [dmin, dmax], M_g = round(n_g d_g / 2) draws."""
    lib = _load()
    n_g, draws = er_params(G, seed, nmin, nmax, dmin, dmax)
    col = np.empty(max(int(2 * draws.sum()), 1), dtype=np.int32)
    rp = np.empty(int(n_g.sum()) + G, dtype=np.int32)
    m_g = np.empty(G, dtype=np.int64)
    lib.graphgen_er_fill(G, seed, _ptr(n_g), _ptr(draws), _ptr(col), _ptr(rp), _ptr(m_g))
    edge_off = np.empty(G + 1, dtype=np.int64)
    lib.graphgen_er_pack(G, _ptr(draws), _ptr(m_g), _ptr(col), _ptr(edge_off))
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(n_g, out=vtx_off[1:])
    m = int(edge_off[G])
    return Batch(vtx_off, edge_off, rp, col[:m].copy())


def trace(R: int, seed: int = 5, rate: float = 2000.0, emin: float = 1e3, emax: float = 5e7):
    """Serving trace of R requests (arrival time s, kind 0=R-MAT 1=lattice,
    scale-or-side, edge factor, keep probability, per-request seed)."""
    t = np.empty(R, dtype=np.float64)
    kind = np.empty(R, dtype=np.int32)
    size = np.empty(R, dtype=np.int64)
    ef = np.empty(R, dtype=np.int32)
    p = np.empty(R, dtype=np.float64)
    rs = np.empty(R, dtype=np.uint64)
    _load().graphgen_trace(R, seed, rate, emin, emax, _ptr(t), _ptr(kind), _ptr(size), _ptr(ef), _ptr(p), _ptr(rs))
    return dict(t=t, kind=kind, size=size, ef=ef, p=p, seed=rs)


def trace_graph(tr, i: int):
    """Materialise request i of a trace as (rp int64, ci int32)."""
    seed = int(tr["seed"][i]) & 0x7FFFFFFFFFFFFFFF
    if int(tr["kind"][i]) == 0:
        return rmat(int(tr["size"][i]), int(tr["ef"][i]), seed=seed)
    return grid(int(tr["size"][i]), float(tr["p"][i]), 0, seed=seed)


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def rmat_s16():
    """R-MAT scale 16 (65,536 vertices), edge factor 16, seed 1, int32-sized."""
    return rmat(16, 16, seed=1)


def grid_4096():
    """4096 x 4096 lattice, p = 0.55, plus 1,000,000 isolated vertices, seed 2."""
    return grid(4096, 0.55, extra=1_000_000, seed=2)


def rmat_s26():
    """R-MAT scale 26 (67,108,864 vertices), edge factor 16, ids permuted (seed 3)."""
    return rmat(26, 16, seed=3, permute=True)


def rmat_s25_ef8():
    """R-MAT scale 25, edge factor 8, ids permuted (seed 3): the profiling
    case (its grandparent vector, 134 MB, exceeds L2; ~2.5 GB on the device)."""
    return rmat(25, 8, seed=3, permute=True)


WORKLOADS = {
    "rmat_s16": rmat_s16,
    "rmat_s25_ef8_perm": rmat_s25_ef8,
    "grid_4096_p055_iso1M": grid_4096,
    "rmat_s26_perm": rmat_s26,
}

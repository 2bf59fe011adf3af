// variants.cuh -- device code of the two alternatives to the default
// FastSV iteration (single graph, sm_103a):
//
// 1. The convergence ablation of Section 5.2 ("Speed of convergence"): the
//    simplified SV algorithm (Algorithm 1, Section 2.4) with the optimizations of
//    Sections 3.1-3.4 added one at a time.
//      sv1  Algorithm 1: tree hooking f_next[f[u]] <- f[v] over the edges
//           whose f[u] is a root (f[u] == f[f[u]]) and f[v] < f[u], the
//           smallest value kept; f <- f_next; shortcutting f <- f[f];
//           stop when f is unchanged
//      sv2  sv1 hooking onto the grandparent f[f[v]] (Section 3.1)
//      sv3  sv2 without the root test: stochastic hooking (Section 3.2)
//      sv4  Algorithm 2's loop body, stochastic and aggressive hooking and
//           shortcutting from one f (Section 3.3), stopping when f is
//           unchanged; sv5 (early termination, Section 3.4) is the default
//           iteration itself
//    The neighbour minimum of each row comes from the default SpMV kernel
//    (k2_spmv gathers from the segment's gf pointer, which for sv1 is the
//    parent snapshot p and otherwise the grandparent vector), so every
//    variant shares the merge-path SpMV; the kernels here apply the hooks,
//    the separate shortcut phase of Algorithm 1 and the variant's stopping
//    test.  Every write is a min of values read from vectors that no kernel
//    of the same phase writes, so each iteration is deterministic and equal
//    to the sequential definition.
//
// 2. The asynchronous mode: Section 2.4 remarks that reading and writing one
//    parent vector still yields the connected components, with pointer
//    graphs that depend on the schedule.  One fused kernel per iteration
//    walks the merge-path tiles, takes each row's minimum of the live f[v],
//    hooks f[f[u]] and f[u] onto it and shortcuts f[u] to f[f[u]], all by
//    atomic min on the single vector f.  An iteration that lowers no entry
//    of f read only the final f, so every tree is a star and f is constant
//    along every edge: the component minima.  The labels are exact; the
//    iteration count depends on the schedule.
#pragma once

#include "fastsv_kernels.cuh"

namespace fsv {

// ---------------------------------------------------------------------------
// convergence ablation sv1..sv4
// ---------------------------------------------------------------------------

struct VarPtrs {
    int32_t* f;       // parent vector (the caller's labels)
    int32_t* p;       // snapshot of f at the start of the iteration
    int32_t* g;       // grandparents p[p] of the snapshot; scratch in between
    const int32_t* mngf;  // per-row minimum of the hook source over the neighbours
    unsigned int* changed;  // segment 0's changed counter
    int64_t n;
};

__global__ void kv_iota(int32_t* x, int64_t n) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        x[v] = (int32_t)v;
}

// hooking of one iteration, from the snapshot p and its grandparents g:
//   root_test   only rows whose parent is a root (p[u] == g[u]) hook (sv1, sv2)
//   aggressive  also f[u] <-min min(mngf[u], g[u]): Algorithm 2's aggressive
//               hooking and shortcutting (sv4)
// The tree hook f[p[u]] <-min mngf[u] is a no-op unless mngf[u] < g[u],
// because f[p[u]] starts at p[p[u]] = g[u] and only decreases.
__global__ void __launch_bounds__(256) kv_hook(VarPtrs P, int root_test, int aggressive) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < P.n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t mn = P.mngf[u];
        if (mn == INF) continue;  // no neighbours
        const int32_t pu = P.p[u], gu = P.g[u];
        if (mn < gu && (!root_test || pu == gu)) atomicMin(P.f + pu, mn);
        if (aggressive) {
            const int32_t m2 = mn < gu ? mn : gu;
            if (m2 < pu) atomicMin(P.f + u, m2);
        }
    }
}

// Algorithm 1's shortcutting phase, on the pointer graph after hooking:
// g[u] = f[f[u]] (g is free until the grandparents are recomputed)
__global__ void __launch_bounds__(256) kv_shortcut(VarPtrs P) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < P.n; u += (int64_t)gridDim.x * blockDim.x)
        P.g[u] = P.f[P.f[u]];
}

// end of an iteration: the new f (g after a shortcut phase, else f itself),
// the count of entries that differ from the snapshot (Algorithm 1's "f
// remains unchanged"), and the new snapshot
__global__ void __launch_bounds__(256) kv_commit(VarPtrs P, int from_g) {
    unsigned c = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < P.n; u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t nf = from_g ? P.g[u] : P.f[u];
        c += nf != P.p[u];
        if (from_g) P.f[u] = nf;
        P.p[u] = nf;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(P.changed, c);
}

// grandparents of the new pointer graph
__global__ void __launch_bounds__(256) kv_grand(VarPtrs P) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < P.n; u += (int64_t)gridDim.x * blockDim.x)
        P.g[u] = P.f[P.f[u]];
}

// iteration bookkeeping shared with the default loop (iteration counter,
// trace, convergence, iteration cap, loop condition)
__global__ void __launch_bounds__(256) k_close(Ctx* ctx, cudaGraphConditionalHandle cond, int use_cond) {
    close_iteration(ctx, cond, use_cond);
}

// ---------------------------------------------------------------------------
// asynchronous mode: one fused kernel per iteration on the single vector f
// ---------------------------------------------------------------------------

// loads of the parent vector that other threads lower while the kernel runs:
// plain loads (L1 may serve an older value, which can only delay a hook; an
// iteration in which nothing is lowered reads the final values everywhere)
__device__ __forceinline__ int32_t ld_live(const int32_t* p) { return *p; }

// Merge-path tiles as in k2_spmv (phases 1 and 2 are the same walk over row
// ends and entries); the values gathered are the live parents f[v], and
// phase 3 hooks and shortcuts at once.  f is deliberately not __restrict__:
// it is read and lowered by atomics in the same kernel.  The counter receives, per tile, the
// number of rows whose processing lowered some entry of f (at most one per
// row and tile, so it cannot wrap).
// shared memory of k_async: row ends, row minima, gathered values of a tile
template <int THREADS, int ITEMS>
constexpr int async_smem_bytes() {
    return (2 * (THREADS * ITEMS + 1) + THREADS * ITEMS) * (int)sizeof(int32_t);
}

template <typename RP, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 5) k_async(Ctx* __restrict__ ctx) {
    constexpr int TILE = THREADS * ITEMS;
    extern __shared__ int32_t smem[];
    int32_t* s_rowend = smem;                // row ends (tile-relative)
    int32_t* s_min = smem + (TILE + 1);      // row minima over the tile's entries
    int32_t* s_val = smem + 2 * (TILE + 1);  // live f[col_idx[e]] of the tile's entries
    __shared__ unsigned s_cnt;
    const int tid = threadIdx.x;
    Seg* S = ctx->segs;
    if (!S->active) return;
    const int32_t* __restrict__ tile_row = ctx->k2_tile_row;
    const RP* __restrict__ rp = (const RP*)S->rp;
    int32_t* f = S->f;
    const int64_t n = S->n, m = S->m;
    const int64_t T = S->k2_ntiles;
    if (tid == 0) s_cnt = 0;
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const int64_t d0 = t * TILE;
        const int64_t d1 = min(d0 + (int64_t)TILE, n + m);
        const int64_t x0 = tile_row[t];
        const int64_t x1 = (t + 1 < T) ? (int64_t)tile_row[t + 1] : n;
        // a malformed row_ptr (validation off) can give tiles whose rows run
        // backwards or outnumber their items: skip them, so no index leaves the tile
        if (x1 < x0 || x1 - x0 > d1 - d0) continue;
        const int64_t y0 = d0 - x0, y1 = d1 - x1;
        const int nfull = (int)(x1 - x0);
        const int R = nfull + (x1 < n ? 1 : 0);
        const int E = (int)(y1 - y0);
        const int D = (int)(d1 - d0);
        const RP* __restrict__ rpt = rp + x0 + 1;
        const int32_t* __restrict__ cit = S->ci + y0;
        for (int i = tid; i < R; i += THREADS) {
            int64_t e = rp_at(rpt, i);
            e = (e < y1 ? e : y1) - y0;
            s_rowend[i] = (int32_t)(e < 0 ? 0 : e);
            s_min[i] = INF;
        }
        {
            int32_t c[ITEMS];
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const int j = tid + q * THREADS;
                c[q] = j < E ? ld_stream(cit + j) : -1;
            }
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const int j = tid + q * THREADS;
                if (j < E) s_val[j] = ((uint32_t)c[q] < (uint64_t)n) ? ld_live(f + c[q]) : INF;
            }
        }
        __syncthreads();
        const int k0 = tid * ITEMS;
        int r = -1;
        int32_t acc = INF;
        if (k0 < D) {
            int lo = 0, hi = nfull;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_rowend[mid] + mid < k0)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            r = lo;
            int y = k0 - lo;
            int rend = r < nfull ? s_rowend[r] : 0x7fffffff;
            const int steps = min(ITEMS, D - k0);
            for (int k = 0; k < steps; ++k) {
                if (y >= rend) {
                    if (acc != INF) atomicMin(&s_min[r], acc);
                    acc = INF;
                    ++r;
                    rend = r < nfull ? s_rowend[r] : 0x7fffffff;
                } else {
                    acc = min(acc, s_val[y]);
                    ++y;
                }
            }
        }
        if (acc != INF && r >= 0 && r < R) atomicMin(&s_min[r], acc);
        __syncthreads();
        // phase 3, per row u with row minimum mn: with fu = f[u] and
        // g = f[fu] (loaded for all of a thread's rows first, independent
        // loads), hook the parent f[fu] <-min mn (stochastic; a no-op unless
        // mn < g) and set f[u] <-min min(mn, g) (aggressive hook and
        // shortcut in one).  An iteration without any lowering therefore
        // saw mn >= f[u] on every row and f[f[u]] == f[u] everywhere.
        constexpr int RPT = ITEMS + 1;  // rows per thread: R <= TILE + 1
        int32_t mn[RPT], fu[RPT], g[RPT];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + q * THREADS;
            mn[q] = i < R ? s_min[i] : INF;
            fu[q] = i < R ? ld_live(f + x0 + i) : 0;
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) g[q] = tid + q * THREADS < R ? ld_live(f + fu[q]) : 0;
        unsigned cnt = 0;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int i = tid + q * THREADS;
            if (i >= R) continue;
            bool low = false;
            if (mn[q] < g[q]) low |= atomicMin(f + fu[q], mn[q]) > mn[q];
            const int32_t t = mn[q] < g[q] ? mn[q] : g[q];
            if (t < fu[q]) low |= atomicMin(f + x0 + i, t) > t;
            cnt += low;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if ((tid & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
        __syncthreads();
    }
    if (tid == 0 && s_cnt) atomicAdd(&S->changed, s_cnt);
}

}  // namespace fsv

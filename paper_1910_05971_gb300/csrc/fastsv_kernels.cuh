// fastsv_kernels.cuh -- device code of the FastSV iteration (sm_103a).
//
// Method: Zhang, Azad, Hu, "FastSV: A Distributed-Memory Connected Component
// Algorithm with Fast Convergence" (arXiv:1910.05971), Algorithm 2 (Section 3)
// in the vector form of Algorithm 3 (Section 4.1).
//
// Device state of one graph ("segment"):
//   p   snapshot of the parent vector f at the start of an iteration
//       (read-only while hooking: plays the role of "f" in Algorithm 2)
//   f   the parent vector being updated (plays "f_next"); equal to p at the
//       start of every iteration; every write is an atomic min
//   gf  grandparents p[p] (Algorithm 3's gf), recomputed after each iteration
//   mngf the per-row minimum of gf over the neighbours (Algorithm 3's mngf);
//       kept from one iteration to the next, so an iteration that pushes
//       only from changed vertices (Section 4.2) can update it in place
//
// One iteration = five kernels (graph nodes of one WHILE-loop body):
//   k_iter_begin   clears the loop condition; resets mngf to +inf when the
//                  coming iteration is a full SpMV
//   k2_spmv        mngf[u] = min_{v in N(u)} gf[v] (the (select2nd,min)
//                  SpMV of Algorithm 3).  Work is split by merge-path tiles
//                  over (rows + entries), so every CTA gets the same amount
//                  of work whatever the degree distribution and reads a
//                  contiguous slice of col_idx; a hub row spans several
//                  tiles, whose partial minima merge with an atomic min.
//                  With column blocks, one launch per block of columns, so
//                  the gathers of one launch hit a slice of gf that stays
//                  in L2.
//   k2_push        the sparse alternative (SpMSpV, Section 4.2): only the
//                  vertices whose gf changed last iteration push their new
//                  gf to their neighbours' mngf.  Exact because gf never
//                  increases: the minimum over the unchanged neighbours is
//                  already in mngf.
//   k2_hook        f[p[u]] min= mngf[u]          (stochastic hooking)
//                  f[u] min= min(mngf[u], gf[u]) (aggressive hooking +
//                  shortcutting)
//   k3_grandparent gf'[u] = f[f[u]], count gf' != gf (the termination test of
//                  Section 3.4 / Algorithm 3's ISNE + reduce), gf = gf',
//                  p = f, and collect the changed vertices as the next
//                  frontier.  The last CTA to finish advances every
//                  segment's iteration counter, retires segments whose count
//                  is zero, picks the next iteration's mode (full SpMV or
//                  push) and sets the CUDA-graph WHILE condition.
// Because hooks are atomic mins of values that depend only on (p, gf), the
// result of an iteration does not depend on thread scheduling: the device
// reproduces the sequential pointer graph of Algorithm 2 bit for bit.
#pragma once

#include "fastsv_types.cuh"

namespace fsv {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }
__device__ __forceinline__ int64_t ld_stream(const int64_t* p) { return (int64_t)__ldcs((const long long*)p); }

template <typename RP>
__device__ __forceinline__ int64_t rp_at(const RP* rp, int64_t i) { return (int64_t)rp[i]; }

// number of rows i in [0, n) whose merge-path row-end position rp[i+1] + i is
// < d (rows fully consumed before diagonal d); Merrill & Garland's merge-path
// search specialised to "row ends vs. entry indices".
// Position of staged entry j in shared memory: one padding word after every
// ITEMS entries.  In a merge-path walk the threads of a warp read entries
// about ITEMS words apart, which puts gcd(ITEMS, 32) lanes on one bank (8
// for ITEMS = 8); padded, the stride is ITEMS + 1, odd, and every lane reads
// its own bank.
template <int ITEMS>
__device__ __forceinline__ int stage_at(int j) { return j + j / ITEMS; }

template <typename RP>
__device__ __forceinline__ int64_t merge_path_rows(const RP* rp, int64_t n, int64_t m, int64_t d) {
    int64_t lo = d > m ? d - m : 0;
    int64_t hi = d < n ? d : n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (rp_at(rp, mid + 1) + mid < d)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int segment_of(const Seg* segs, int nsegs, int64_t t, bool k2) {
    int lo = 0, hi = nsegs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int64_t start = k2 ? segs[mid].k2_tile0 : segs[mid].k3_tile0;
        if (start <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// set-up kernels (once per call)
// ---------------------------------------------------------------------------

// workspace pointers owned by the handle, written into the context every call
struct WsPtrs {
    Seg* segs;
    int32_t* k2_seg;
    int32_t* k2_row;
    int32_t* k3_seg;
};

__device__ __forceinline__ void set_ws(Ctx* ctx, const WsPtrs& ws) {
    ctx->segs = ws.segs;
    ctx->k2_tile_seg = ws.k2_seg;
    ctx->k2_tile_row = ws.k2_row;
    ctx->k3_tile_seg = ws.k3_seg;
}

struct SingleParams {
    const void* rp;
    const int32_t* ci;
    int32_t* f;
    int32_t* p;
    int32_t* gf;
    int32_t* mngf;
    int32_t* frontier;       // room for n (segment, vertex) pairs
    int32_t sparse_div;      // 0: sparse iterations off
    int64_t n, m;
    int32_t k2_tile;
    int32_t max_iters;
    int32_t loop_limit;
};

// one graph: segment 0 and the call's scalars
__global__ void k_setup_single(Ctx* ctx, SingleParams prm, WsPtrs ws) {
    set_ws(ctx, ws);
    Seg s;
    s.rp = prm.rp;
    s.ci = prm.ci;
    s.f = prm.f;
    s.p = prm.p;
    s.gf = prm.gf;
    s.n = prm.n;
    s.m = prm.m;
    s.k2_tile0 = 0;
    s.k3_tile0 = 0;
    s.k2_ntiles = prm.m > 0 ? (int32_t)((prm.n + prm.m + prm.k2_tile - 1) / prm.k2_tile) : 0;
    s.k3_ntiles = (int32_t)((prm.n + K3_TILE - 1) / K3_TILE);
    s.active = prm.n > 0;
    s.iters = 0;
    s.status = 0;
    s.converged = 0;
    s.changed = 0;
    s.user = 0;
    s.leader = 0;
    s.mode = 0;
    s.mngf = prm.mngf;
    s.fr_deg = 0;
    s.rowmap = nullptr;
    ws.segs[0] = s;
    ctx->num_segs = 1;
    ctx->k2_tile = prm.k2_tile;
    ctx->k2_total = s.k2_ntiles;
    ctx->k3_total = s.k3_ntiles;
    ctx->max_iters = prm.max_iters;
    ctx->loop_limit = prm.loop_limit;
    ctx->loop_iter = 0;
    ctx->k3_done = 0;
    ctx->any_active = s.active;
    ctx->val_status = 0;
    ctx->sparse_enabled = prm.sparse_div > 0;
    ctx->mode = MODE_DENSE;
    ctx->frontier = prm.frontier;
    ctx->frontier_len = 0;
    ctx->frontier_next = 0;
    ctx->frontier_cap = (unsigned int)(prm.n < 0x7fffffff ? prm.n : 0x7fffffff);
    ctx->frontier_overflow = 0;
    ctx->sparse_div = prm.sparse_div;
    ctx->sparse_iters = 0;
    ctx->blk_chunks = 1;
    for (int i = 0; i < TRACE_LEN; ++i) ctx->sum.trace[i] = 0;
}

struct BatchParams {
    int32_t G;
    const int64_t* vtx_off;
    const int64_t* edge_off;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    int32_t* labels;
    int32_t* p;
    int32_t* gf;
    int32_t* mngf;
    int32_t* frontier;       // room for frontier_cap (segment, vertex) pairs
    int64_t frontier_cap;
    int32_t sparse_div;      // 0: sparse iterations off
    int32_t k2_tile;
    int32_t max_iters;
    int32_t loop_limit;
};

// many graphs: one segment per graph (tile counts; offsets come from k_scan_tiles)
__global__ void k_setup_batched(Ctx* ctx, BatchParams prm, WsPtrs ws) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < prm.G; g += (int64_t)gridDim.x * blockDim.x) {
        int64_t v0 = prm.vtx_off[g], v1 = prm.vtx_off[g + 1];
        int64_t e0 = prm.edge_off[g], e1 = prm.edge_off[g + 1];
        int64_t n = v1 - v0, m = e1 - e0;
        if (n < 0) n = 0;
        if (m < 0) m = 0;
        Seg s;
        s.rp = prm.row_ptr + v0 + g;
        s.ci = prm.col_idx + e0;
        s.f = prm.labels + v0;
        s.p = prm.p + v0;
        s.gf = prm.gf + v0;
        s.n = n;
        s.m = m;
        s.k2_tile0 = 0;
        s.k3_tile0 = 0;
        s.k2_ntiles = (m > 0 && n > 0) ? (int32_t)((n + m + prm.k2_tile - 1) / prm.k2_tile) : 0;
        s.k3_ntiles = (int32_t)((n + K3_TILE - 1) / K3_TILE);
        s.active = n > 0;
        s.iters = 0;
        s.status = 0;
        s.converged = n == 0;
        s.changed = 0;
        s.user = (int32_t)g;
        s.leader = (int32_t)g;
        s.mode = 0;
        s.mngf = prm.mngf + v0;
        s.fr_deg = 0;
        s.rowmap = nullptr;
        ws.segs[g] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        set_ws(ctx, ws);
        ctx->num_segs = prm.G;
        ctx->k2_tile = prm.k2_tile;
        ctx->max_iters = prm.max_iters;
        ctx->loop_limit = prm.loop_limit;
        ctx->loop_iter = 0;
        ctx->k3_done = 0;
        ctx->val_status = 0;
        ctx->sparse_enabled = prm.sparse_div > 0;
        ctx->mode = MODE_DENSE;
        ctx->frontier = prm.frontier;
        ctx->frontier_len = 0;
        ctx->frontier_next = 0;
        ctx->frontier_cap = (unsigned int)(prm.frontier_cap < 0x7fffffff ? prm.frontier_cap : 0x7fffffff);
        ctx->frontier_overflow = 0;
        ctx->sparse_div = prm.sparse_div;
        ctx->sparse_iters = 0;
        ctx->blk_chunks = 1;
        for (int i = 0; i < TRACE_LEN; ++i) ctx->sum.trace[i] = 0;
    }
}

// exclusive prefix sums of the per-segment tile counts (one CTA of 1024
// threads, each owning a contiguous chunk of segments)
__global__ void __launch_bounds__(1024) k_scan_tiles(Ctx* ctx) {
    __shared__ long long s2[1024], s3[1024];
    __shared__ int s_any[1024];
    const int G = ctx->num_segs;
    Seg* segs = ctx->segs;
    const int tid = threadIdx.x;
    const int chunk = (G + 1023) / 1024;
    const int b = tid * chunk, e = min(G, b + chunk);
    long long a2 = 0, a3 = 0;
    int any = 0;
    // only active segments get tiles (a pool keeps retired slots in place)
    for (int g = b; g < e; ++g) {
        if (!segs[g].active) continue;
        a2 += segs[g].k2_ntiles;
        a3 += segs[g].k3_ntiles;
        any = 1;
    }
    s2[tid] = a2;
    s3[tid] = a3;
    s_any[tid] = any;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        long long v2 = tid >= off ? s2[tid - off] : 0, v3 = tid >= off ? s3[tid - off] : 0;
        int va = tid >= off ? s_any[tid - off] : 0;
        __syncthreads();
        s2[tid] += v2;
        s3[tid] += v3;
        s_any[tid] |= va;
        __syncthreads();
    }
    long long o2 = s2[tid] - a2, o3 = s3[tid] - a3;
    for (int g = b; g < e; ++g) {
        segs[g].k2_tile0 = o2;
        segs[g].k3_tile0 = o3;
        if (!segs[g].active) continue;
        o2 += segs[g].k2_ntiles;
        o3 += segs[g].k3_ntiles;
    }
    if (tid == 1023) {
        ctx->k2_total = s2[1023];
        ctx->k3_total = s3[1023];
        ctx->any_active = s_any[1023];
    }
}

// merge-path start row of every hooking tile, and the segment of every tile
template <typename RP>
__global__ void k_partition(Ctx* ctx) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const Seg* segs = ctx->segs;
    const int G = ctx->num_segs;
    const int64_t tile = ctx->k2_tile;
    for (int64_t t = t0; t < ctx->k2_total; t += stride) {
        int s = segment_of(segs, G, t, true);
        const Seg& S = segs[s];
        int64_t d = (t - S.k2_tile0) * tile;
        ctx->k2_tile_seg[t] = s;
        ctx->k2_tile_row[t] = (int32_t)merge_path_rows((const RP*)S.rp, S.n, S.m, d);
    }
    for (int64_t t = t0; t < ctx->k3_total; t += stride) ctx->k3_tile_seg[t] = segment_of(segs, G, t, false);
}

// f = p = gf = local identity (Algorithm 2: f[u] <- u; Algorithm 3: gf = dup(f))
// for every active segment that has not run an iteration yet
__global__ void k_init_state(Ctx* ctx) {
    const int64_t total = ctx->k3_total;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const Seg& S = ctx->segs[ctx->k3_tile_seg[t]];
        if (!S.active || S.iters != 0) continue;
        int64_t v0 = (t - S.k3_tile0) * K3_TILE;
        int64_t v1 = min(v0 + K3_TILE, S.n);
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            S.f[v] = (int32_t)v;
            S.p[v] = (int32_t)v;
            S.gf[v] = (int32_t)v;
        }
    }
}

// CSR validation: row_ptr[0] = 0, non-decreasing, row_ptr[n] = m; every
// neighbour id in [0, n); with check_sym, (v,u) present for every (u,v)
// (binary search, rows must be sorted).  Sets ctx->val_status bits.
template <typename RP>
__global__ void k_validate(Ctx* ctx, int check_sym) {
    const int64_t total = ctx->k3_total;
    int32_t bad = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const Seg& S = ctx->segs[ctx->k3_tile_seg[t]];
        const RP* rp = (const RP*)S.rp;
        int64_t v0 = (t - S.k3_tile0) * K3_TILE;
        int64_t v1 = min(v0 + K3_TILE, S.n);
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            int64_t a = rp_at(rp, v), b = rp_at(rp, v + 1);
            if (v == 0 && a != 0) bad |= DEV_ERR_BAD_ROWPTR;
            if (b < a || a < 0 || b > S.m) {
                bad |= DEV_ERR_BAD_ROWPTR;
                continue;
            }
            if (v + 1 == S.n && b != S.m) bad |= DEV_ERR_BAD_ROWPTR;
            for (int64_t e = a; e < b; ++e) {
                int32_t w = S.ci[e];
                if (w < 0 || w >= S.n) {
                    bad |= DEV_ERR_BAD_COLIDX;
                    break;
                }
                if (check_sym) {
                    int64_t lo = rp_at(rp, w), hi = rp_at(rp, w + 1);
                    if (hi < lo || lo < 0 || hi > S.m) {
                        bad |= DEV_ERR_BAD_ROWPTR;
                        break;
                    }
                    while (lo < hi) {
                        int64_t mid = (lo + hi) >> 1;
                        if (S.ci[mid] < (int32_t)v)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    if (lo >= rp_at(rp, w + 1) || S.ci[lo] != (int32_t)v) bad |= DEV_ERR_ASYMMETRIC;
                }
            }
        }
    }
    if (bad) atomicOr(&ctx->val_status, bad);
}

// ---------------------------------------------------------------------------
// Column blocking of one graph (set-up, once per call)
//
// Hooking gathers gf[col_idx[e]] at random positions.  When gf is larger
// than L2 most gathers miss.  Splitting the columns into nb ranges of 2^shift
// ids and running one SpMV pass per range keeps every pass's gathers inside
// an L2-resident slice of gf.  A row's minimum over all its entries is the
// minimum of its per-range minima and every hook is a min, so hooking with
// each range's minimum gives exactly the f of the unsplit SpMV.  (This is the
// single-GPU counterpart of the 2-D distribution of A in Section 4.2, where
// each process column owns a range of columns.)
//
// Layout of the block copy (compressed rows: a block lists only the rows that
// have entries in it).  The copy is cut along the merge-path tiles of the
// graph's own CSR (the first iteration's tiles, BUILD_TILE items each), and
// the tiles are grouped into C chunks of consecutive tiles (C = 1, or one
// chunk per piece in which col_idx arrives from host memory, so that a chunk
// is copied as soon as its entries are there).  Inside a tile, a "run" is a
// maximal sequence of consecutive entries of one row whose columns fall in
// one block; when rows are sorted by column a row has exactly one run per
// block it touches.  Chunk c occupies the entries [Y_c, Y_{c+1}) of colB
// (the same entries as in the CSR), block after block; block b of chunk c
// holds, tile after tile, the tile's runs of block b in tile order (a stable
// partition of the tile's entries by block):
//   colB[ebase_cb + ...]          the entries (global column ids)
//   rowsB[pbase_cb + i]           global row of run i; bit 31 set when the
//                                 row may have another run in the block (the
//                                 row crosses a tile boundary, or the tile's
//                                 rows are not sorted by block), so its
//                                 partial minimum must merge atomically
//   endsB[pbase_cb + s + i + 1]   end of run i inside the block's entries of
//                                 the chunk, s = c nb + b (endsB[pbase_cb +
//                                 s] = 0): every (chunk, block) is a CSR over
//                                 its runs, walked by the same merge-path
//                                 SpMV as the graph itself.
// The first iteration's SpMV counts every tile's entries and runs per block;
// an exclusive scan over a chunk's tiles gives every (tile, block) its
// offsets, and the chunk's totals place its blocks (ChunkLayout).
// ---------------------------------------------------------------------------

constexpr int32_t ROW_SHARED = (int32_t)0x80000000u;  // rowsB flag: merge this run's minimum atomically

__device__ __forceinline__ int col_block(int32_t c, int shift, int nb) {
    int b = (int)((uint32_t)c >> shift);
    return b < nb ? b : nb - 1;
}

constexpr int BUILD_THREADS = 128;  // CTA size and items per thread of the block-split kernel
constexpr int BUILD_ITEMS = 8;
constexpr int BUILD_TILE = BUILD_THREADS * BUILD_ITEMS;

// The block copy: for every tile of segment 0 (the tiles the first
// iteration counted), a stable partition of its entries by column block.
// One warp per tile walks the tile's entries in rounds of 32 (a batch of
// rounds' column ids loaded at once); lanes of one block find each other
// with a match, rank themselves by the lanes before them, and write their
// entries at the block's running position (the tile's scanned offset,
// advanced by the group leader after every round).  Run starts are noted in
// shared memory; after every batch one pass over them (lanes over runs)
// finds each run's row from the row-start bitmap and writes the run's row
// and, as the end of the block's previous run, its position.  The end of
// every block's last run is its entry count.
constexpr int SPLIT_WARPS = 4;
constexpr int SPLIT_THREADS = 32 * SPLIT_WARPS;
constexpr int SPLIT_BATCH = 8;                  // rounds whose column ids are loaded together
constexpr int SPLIT_RUNS = 32 * SPLIT_BATCH;    // runs a batch can start

// This launch copies chunk `chunk` (tiles [range[chunk], range[chunk + 1]),
// or every tile when range is null); p_total is the length of rowsB and
// endsB: no write goes at or beyond it (the host checks that the runs fit).
template <typename RP>
__global__ void __launch_bounds__(32 * SPLIT_WARPS)
    k_block_split(const Ctx* __restrict__ ctx, const ChunkLayout* __restrict__ lay, int chunk, int nb, int shift,
                  int64_t T1, const int64_t* __restrict__ range, const int32_t* __restrict__ cnt,
                  int32_t* __restrict__ colB, int32_t* __restrict__ rowsB, int32_t* __restrict__ endsB,
                  int64_t m_total, int64_t p_total) {
    __shared__ int16_t s_rowof[SPLIT_WARPS][BUILD_TILE];    // row starting at a position (valid where s_rs is set)
    __shared__ unsigned s_rs[SPLIT_WARPS][BUILD_TILE / 32];  // bit j: entry j is the first entry of a row
    __shared__ int32_t s_pos[SPLIT_WARPS][MAX_COL_BLOCKS];   // next entry position inside each block
    __shared__ int32_t s_run[SPLIT_WARPS][MAX_COL_BLOCKS];   // next run index inside each block
    __shared__ int32_t s_rp[SPLIT_WARPS][SPLIT_RUNS];        // a batch's runs: position inside the block,
    __shared__ int32_t s_ri[SPLIT_WARPS][SPLIT_RUNS];        //   index among the block's runs,
    __shared__ int16_t s_rj[SPLIT_WARPS][SPLIT_RUNS];        //   first entry in the tile,
    __shared__ int8_t s_rb[SPLIT_WARPS][SPLIT_RUNS];         //   block
    __shared__ long long s_eb[MAX_COL_BLOCKS], s_pb[MAX_COL_BLOCKS];
    const Seg S0 = ctx->segs[0];
    const ChunkLayout& L = lay[chunk];
    const int sub0 = chunk * nb;  // run CSRs of earlier (chunk, block) pairs: one leading slot each
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    if ((int)threadIdx.x < nb) {
        s_eb[threadIdx.x] = L.ebase[threadIdx.x];
        s_pb[threadIdx.x] = L.pbase[threadIdx.x] + sub0;  // + b: endsB index of run 0; - sub0: rowsB index
        if (blockIdx.x == 0) {  // the end of the block's last run
            const int b = threadIdx.x;
            const int64_t pb = L.pbase[b + 1] - L.pbase[b];
            const int64_t at = L.pbase[b] + sub0 + b + pb;
            if (at < p_total) endsB[at] = (int32_t)(L.ebase[b + 1] - L.ebase[b]);
        }
    }
    __syncthreads();
    const RP* __restrict__ rp = (const RP*)S0.rp;
    const int32_t* __restrict__ ci = S0.ci;
    const int64_t n = S0.n, m = S0.m, T = S0.k2_ntiles;
    const int32_t* __restrict__ tile_row = ctx->k2_tile_row + S0.k2_tile0;
    unsigned* rsw = s_rs[w];
    int16_t* rowof = s_rowof[w];
    const int64_t t_end = range ? min(range[chunk + 1], T) : T;
    for (int64_t t = (range ? range[chunk] : 0) + (int64_t)blockIdx.x * SPLIT_WARPS + w; t < t_end;
         t += (int64_t)gridDim.x * SPLIT_WARPS) {
        const int64_t d0 = t * BUILD_TILE, d1 = min(d0 + BUILD_TILE, n + m);
        const int64_t x0 = tile_row[t];
        const int64_t x1 = t + 1 < T ? (int64_t)tile_row[t + 1] : n;
        // a malformed row_ptr (validation off) can give tiles whose rows run
        // backwards or outnumber their items: skip them, so no index leaves the tile
        if (x1 < x0 || x1 - x0 > d1 - d0) continue;
        const int64_t y0 = d0 - x0, y1 = d1 - x1;
        const int nfull = (int)(x1 - x0);
        const int E = (int)(y1 - y0);
        if (E <= 0) continue;
        rsw[lane] = 0u;
        if (lane < nb) {
            s_pos[w][lane] = cnt[(int64_t)lane * T1 + t];
            s_run[w][lane] = cnt[(int64_t)(nb + lane) * T1 + t];
        }
        const bool first_whole = rp_at(rp, x0) >= y0;  // row x0 starts inside the tile
        __syncwarp();
        // the first entry of every row that starts inside the tile: row i + 1
        // starts where row i ends (rows without entries start nowhere)
        for (int i = lane; i <= nfull; i += 32) {
            int64_t st = i == 0 ? (first_whole ? y0 : y1) : rp_at(rp, x0 + i);
            int64_t en = i < nfull ? rp_at(rp, x0 + 1 + i) : y1;
            st = (st < y1 ? st : y1) - y0;
            en = (en < y1 ? en : y1) - y0;
            if (st >= 0 && st < en) {
                atomicOr(&rsw[st >> 5], 1u << (st & 31));
                rowof[st] = (int16_t)i;
            }
        }
        __syncwarp();
        int prev_b = -1;  // block of the entry before the round
        bool desc = false;
        for (int base = 0; base < E; base += 32 * SPLIT_BATCH) {
            int32_t cv[SPLIT_BATCH];
#pragma unroll
            for (int k = 0; k < SPLIT_BATCH; ++k) {
                const int j = base + 32 * k + lane;
                cv[k] = j < E ? ld_stream(ci + y0 + j) : 0;
            }
            int nruns = 0;  // runs started in this batch
#pragma unroll
            for (int k = 0; k < SPLIT_BATCH; ++k) {
                const int j = base + 32 * k + lane;
                if (j - lane >= E) break;  // warp-uniform
                const bool valid = j < E;
                const int32_t c = cv[k];
                const int b = valid ? col_block(c, shift, nb) : 0;
                int pb = __shfl_up_sync(0xffffffffu, b, 1);
                if (lane == 0) pb = prev_b;
                prev_b = __shfl_sync(0xffffffffu, b, 31);
                const bool row_first = valid && (j == 0 || ((rsw[j >> 5] >> (j & 31)) & 1u));
                const bool rs = valid && (row_first || pb != b);
                desc |= valid && !row_first && pb > b;
                const unsigned grp = __match_any_sync(0xffffffffu, valid ? b : 64 + lane);
                const unsigned rsb = __ballot_sync(0xffffffffu, rs);
                const int p = s_pos[w][b] + __popc(grp & lt);
                if (valid) {
                    const int64_t at = s_eb[b] + p;
                    if (at < m_total) colB[at] = c;
                    if (rs) {
                        const int k2 = nruns + __popc(rsb & lt);
                        s_rp[w][k2] = p;
                        s_ri[w][k2] = s_run[w][b] + __popc(grp & rsb & lt);
                        s_rj[w][k2] = (int16_t)j;
                        s_rb[w][k2] = (int8_t)b;
                    }
                }
                nruns += __popc(rsb);
                __syncwarp();
                if (valid && (__ffs(grp) - 1) == lane) {
                    s_pos[w][b] += __popc(grp);
                    s_run[w][b] += __popc(grp & rsb);
                }
                __syncwarp();
            }
            // the batch's runs: row (the last row start at or before the
            // run's first entry; none: the row that began before the tile)
            for (int k2 = lane; k2 < nruns; k2 += 32) {
                const int j = s_rj[w][k2], b = s_rb[w][k2];
                int wd = j >> 5;
                unsigned bits = rsw[wd] & (0xffffffffu >> (31 - (j & 31)));
                while (!bits && wd > 0) bits = rsw[--wd];
                const int row = bits ? rowof[wd * 32 + 31 - __clz(bits)] : 0;
                const bool shared = (row == 0 && !first_whole) || row >= nfull;
                const int64_t pi = s_pb[b] + s_ri[w][k2];
                if (pi + b < p_total) {
                    rowsB[pi - sub0] = (int32_t)(x0 + row) | (shared ? ROW_SHARED : 0);
                    endsB[pi + b] = s_rp[w][k2];  // the block's previous run ends where this one starts
                }
            }
            __syncwarp();
        }
        // a row whose block id decreases: its block may repeat inside the
        // tile, so every run of this tile merges atomically
        if (__any_sync(0xffffffffu, desc)) {
            for (int b = 0; b < nb; ++b) {
                const int r0 = cnt[(int64_t)(nb + b) * T1 + t], r1 = s_run[w][b];
                for (int i = r0 + lane; i < r1; i += 32)
                    if (s_pb[b] + i < p_total) rowsB[s_pb[b] - sub0 + i] |= ROW_SHARED;
            }
        }
        __syncwarp();
    }
}

// exclusive scan of rows of int32 (row r at in + r L), over the tiles of
// one chunk (columns [range[rc], range[rc + 1]) of every row, or [0, L) when
// range is null), in pieces of SCAN_CHUNK: piece sums, per-row scan of the
// sums (whose total is the chunk's), apply.  Launched with `pieces` CTAs per
// row, enough for any chunk; CTAs past the chunk's end do nothing.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int block_exclusive_scan(int v, int* s_warp, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = s;
    }
    __syncthreads();
    const int before = (w > 0 ? s_warp[w - 1] : 0) + x - v;
    if (total) *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__device__ __forceinline__ void scan_bounds(const int64_t* range, int rc, int64_t L, int64_t& t0, int64_t& t1) {
    t0 = range ? range[rc] : 0;
    t1 = range ? range[rc + 1] : L;
    t1 = t1 < L ? t1 : L;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_chunk_sums(const int32_t* in, int64_t L, int pieces,
                                                                 int32_t* sums, const int64_t* range, int rc) {
    __shared__ int s_warp[32];
    const int row = blockIdx.x / pieces, c = blockIdx.x % pieces;
    int64_t t0, t1;
    scan_bounds(range, rc, L, t0, t1);
    const int32_t* p = in + (int64_t)row * L;
    const int64_t base = t0 + (int64_t)c * SCAN_CHUNK;
    int acc = 0;
    if (base < t1)
        for (int i = threadIdx.x; i < SCAN_CHUNK; i += SCAN_THREADS) {
            int64_t j = base + i;
            if (j < t1) acc += p[j];
        }
    int total = 0;
    block_exclusive_scan(acc, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// one CTA per row; totals[row]: the row's sum over the chunk
__global__ void __launch_bounds__(1024) k_scan_sums(int32_t* sums, int pieces, int32_t* totals) {
    __shared__ int s_warp[32];
    int32_t* p = sums + (int64_t)blockIdx.x * pieces;
    int carry = 0;
    for (int base = 0; base < pieces; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < pieces ? p[i] : 0;
        int total = 0;
        int ex = block_exclusive_scan(v, s_warp, &total);
        if (i < pieces) p[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const int32_t* in, int32_t* out, int64_t L, int pieces,
                                                            const int32_t* sums, const int64_t* range, int rc) {
    __shared__ int s_warp[32];
    const int row = blockIdx.x / pieces, c = blockIdx.x % pieces;
    int64_t t0, t1;
    scan_bounds(range, rc, L, t0, t1);
    if (t0 + (int64_t)c * SCAN_CHUNK >= t1) return;  // CTA-uniform: past the chunk's end
    const int32_t* p = in + (int64_t)row * L;
    int32_t* q = out + (int64_t)row * L;
    const int64_t base = t0 + (int64_t)c * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int acc = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t j = base + k;
        v[k] = j < t1 ? p[j] : 0;
        acc += v[k];
    }
    int run = sums[blockIdx.x] + block_exclusive_scan(acc, s_warp, nullptr);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t j = base + k;
        if (j < t1) q[j] = run;
        run += v[k];
    }
}

// chunk `chunk`'s blocks from its scanned totals (tot: entries per block,
// then runs per block): its entries start where its first tile's do, its
// runs where the previous chunk's end
__global__ void k_chunk_layout(const Ctx* __restrict__ ctx, const int32_t* __restrict__ tot, int nb,
                               const int64_t* __restrict__ range, int chunk, ChunkLayout* lay) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const Seg& S = ctx->segs[0];
    const int64_t T = S.k2_ntiles;
    const int64_t t0 = range ? range[chunk] : 0;
    int64_t e = t0 < T ? t0 * ctx->k2_tile - ctx->k2_tile_row[S.k2_tile0 + t0] : S.m;
    int64_t p = chunk > 0 ? lay[chunk - 1].pbase[nb] : 0;
    ChunkLayout& L = lay[chunk];
    for (int b = 0; b < nb; ++b) {
        L.ebase[b] = e;
        L.pbase[b] = p;
        e += (uint32_t)tot[b];
        p += (uint32_t)tot[nb + b];
    }
    L.ebase[nb] = e;
    L.pbase[nb] = p;
}

// for the host: out[0] the end of the last chunk's entries (m for a valid
// CSR), out[1] the runs of all chunks, out[2] 1 when every chunk's entries
// end where the next chunk's begin
__global__ void k_chunk_check(const ChunkLayout* __restrict__ lay, int chunks, int nb, int64_t* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t ok = 1;
    for (int c = 0; c + 1 < chunks; ++c) ok &= lay[c].ebase[nb] == lay[c + 1].ebase[0];
    out[0] = lay[chunks - 1].ebase[nb];
    out[1] = lay[chunks - 1].pbase[nb];
    out[2] = ok;
}

// segments 1 .. nb C: the column blocks of graph 0, chunk by chunk (block b
// of chunk c is segment 1 + b C + c, so a block's segments are adjacent;
// compressed rows: the runs are the rows, rowsB maps them to the graph's
// rows); graph 0 keeps only its grandparent tiles
__global__ void __launch_bounds__(256) k_setup_blocks(Ctx* ctx, const ChunkLayout* __restrict__ lay, int chunks, int nb,
                                                      const int32_t* colB, const int32_t* rowsB, const int32_t* endsB,
                                                      int32_t k2_tile) {
    Seg* segs = ctx->segs;
    const Seg g = segs[0];
    for (int i = threadIdx.x; i < nb * chunks; i += blockDim.x) {
        const int c = i / nb, b = i % nb;
        const ChunkLayout& L = lay[c];
        const int64_t pb = L.pbase[b + 1] - L.pbase[b];
        const int64_t mb = L.ebase[b + 1] - L.ebase[b];
        Seg s = g;
        s.rp = endsB + L.pbase[b] + i;  // one leading slot per earlier (chunk, block) pair
        s.ci = colB + L.ebase[b];
        s.rowmap = rowsB + L.pbase[b];
        s.n = pb;
        s.m = mb;
        s.k2_ntiles = mb > 0 ? (int32_t)((pb + mb + k2_tile - 1) / k2_tile) : 0;
        s.k3_ntiles = 0;
        s.active = 1;
        s.leader = 0;
        s.user = b;
        segs[1 + b * chunks + c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        segs[0].k2_ntiles = 0;
        ctx->num_segs = 1 + nb * chunks;
        ctx->blk_chunks = chunks;
        ctx->k2_tile = k2_tile;
        ctx->loop_iter = 0;  // an iteration run before the blocks is not the device loop's
    }
}

// ---------------------------------------------------------------------------
// K2: SpMV (select2nd, min) fused with the three hooks
// ---------------------------------------------------------------------------

// first kernel of every iteration: resets the loop condition to "stop" (only
// the last CTA of k3_grandparent sets it back to "continue" when work
// remains, so a device loop can never outlive its bookkeeping), and before a
// full SpMV sets mngf to INF for every active graph that runs one
__global__ void k_iter_begin(Ctx* __restrict__ ctx, cudaGraphConditionalHandle cond, int use_cond) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    if (!(ctx->mode & MODE_DENSE)) return;
    const int64_t total = ctx->k3_total;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const Seg& S = ctx->segs[ctx->k3_tile_seg[t]];
        if (!S.active || S.mode != 0) continue;  // a pushing graph keeps its mngf
        const int64_t v0 = (t - S.k3_tile0) * K3_TILE;
        const int64_t v1 = min(v0 + K3_TILE, S.n);
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) S.mngf[v] = INF;
    }
}

// a1, full iteration: mngf[u] = min_{v in N(u)} gf[v] -- the (select2nd,min)
// SpMV of Section 4.1.  One CTA of THREADS threads handles one merge-path
// tile of THREADS*ITEMS items (row ends + entries) at a time; a row split
// over tiles (or over column blocks) contributes one partial minimum per
// tile, merged by atomic min into mngf.
//
// block < 0: every tile of every segment (no column blocking).  block >= 0:
// only the tiles of column block `block` of graph 0, whose rows are the
// block's runs (rowmap gives each run's graph row); every run's minimum
// merges by a fire-and-forget atomic min (no load round trip in the tile).
// A launch over one segment (a column block, or a single graph) reads the
// segment's fields once, and every tile reads the next tile's merge-path
// start rows ahead, so a tile's only waits are its column ids and gathers.
template <typename RP, int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 1536 / THREADS) k2_spmv(Ctx* __restrict__ ctx, int block) {
    constexpr int TILE = THREADS * ITEMS;
    if (!(ctx->mode & MODE_DENSE)) return;
    extern __shared__ int32_t smem[];
    int32_t* s_rowend = smem;                 // local end offset of each row in the tile
    int32_t* s_mngf = smem + (TILE + 1);      // per-row minimum over the tile's entries
    int32_t* s_val = smem + 2 * (TILE + 1);   // gf[col_idx[e]] for the tile's entries (at stage_at)
    const int tid = threadIdx.x;
    const int32_t* __restrict__ tile_seg = ctx->k2_tile_seg;
    const int32_t* __restrict__ tile_row = ctx->k2_tile_row;
    const Seg* __restrict__ segs = ctx->segs;
    const int64_t total = ctx->k2_total;
    int64_t t_begin = 0, T = total;
    const int chunks = ctx->blk_chunks;  // segments of one column block
    if (block >= 0) {
        if (1 + (block + 1) * chunks > ctx->num_segs) return;
        const Seg& first = segs[1 + block * chunks];
        const Seg& last = segs[(block + 1) * chunks];
        t_begin = first.k2_tile0;
        T = last.k2_tile0 + last.k2_ntiles;
    }
    const bool merge = block >= 0;
    // one graph for the whole launch (a column block, or a single graph):
    // its state is checked once; with one segment (a block copied as one
    // chunk, or a single graph) no tile looks its segment up either
    const bool one_state = block >= 0 || ctx->num_segs == 1;
    const bool one_seg = (block >= 0 && chunks == 1) || ctx->num_segs == 1;
    const int32_t seg0 = block >= 0 ? 1 + block * chunks : 0;
    bool ident1 = false;
    int64_t ncol1 = 0;
    if (one_state) {
        const Seg& L = segs[segs[seg0].leader];
        if (!L.active || L.mode != 0) return;
        ident1 = L.iters == 0;
        ncol1 = L.n;
    }
    int64_t t = t_begin + blockIdx.x;
    int32_t xa = t < T ? tile_row[t] : 0, xb = t + 1 < total ? tile_row[t + 1] : 0;

    for (; t < T; t += gridDim.x) {
        // this tile's merge-path start rows, and the next tile's, read ahead
        const int32_t xr0 = xa, xr1 = xb;
        const int64_t tn = t + gridDim.x;
        if (tn < T) {
            xa = tile_row[tn];
            xb = tn + 1 < total ? tile_row[tn + 1] : 0;
        }
        const Seg* S = segs + seg0;
        bool ident = ident1;
        int64_t ncol = ncol1;
        if (!one_seg) {
            S = segs + tile_seg[t];
            if (!one_state) {
                const Seg& L = segs[S->leader];
                if (!L.active || L.mode != 0) continue;
                ident = L.iters == 0;
                ncol = L.n;
            }
        }
        const RP* __restrict__ rp = (const RP*)S->rp;
        const int32_t* __restrict__ gf = S->gf;
        int32_t* mngf = S->mngf;
        const int64_t n = S->n, m = S->m;
        const int64_t lt = t - S->k2_tile0;
        const int64_t d0 = lt * TILE;
        const int64_t d1 = min(d0 + (int64_t)TILE, n + m);
        const int64_t x0 = xr0;
        const int64_t x1 = (lt + 1 < S->k2_ntiles) ? (int64_t)xr1 : n;
        // a malformed row_ptr (validation off) can give tiles whose rows run
        // backwards or outnumber their items: skip them, so no index leaves the tile
        if (x1 < x0 || x1 - x0 > d1 - d0) continue;
        const int64_t y0 = d0 - x0, y1 = d1 - x1;
        const int nfull = (int)(x1 - x0);            // rows whose end lies in this tile
        const int R = nfull + (x1 < n ? 1 : 0);       // plus the row still open at the tile end
        const int E = (int)(y1 - y0);                 // entries in this tile
        const int D = (int)(d1 - d0);
        const RP* __restrict__ rpt = rp + x0 + 1;     // row ends of the tile's rows
        const int32_t* __restrict__ cit = S->ci + y0; // the tile's entries

        // phase 1: row ends, and the gathered grandparents of the tile's
        // entries (in the graph's first iteration gf is still the identity:
        // every vertex its own root, so gf[v] = v and nothing is gathered)
        for (int i = tid; i < R; i += THREADS) {
            int64_t e = rp_at(rpt, i);
            e = (e < y1 ? e : y1) - y0;
            s_rowend[i] = (int32_t)(e < 0 ? 0 : e);
            s_mngf[i] = INF;
        }
        {
            int32_t c[ITEMS];
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const int j = tid + q * THREADS;
                c[q] = j < E ? ld_stream(cit + j) : -1;
            }
            // entry tid + q THREADS sits at stage_at(tid) + q (THREADS + THREADS / ITEMS)
            const int sb = stage_at<ITEMS>(tid);
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const int j = tid + q * THREADS;
                // gathers cached in L2 only: a gathered sector is rarely reused by
                // the same SM, and skipping L1 allocation measured 4.5% faster on
                // the column-blocked SpMV at R-MAT scale 26 (9.86 vs 10.32 ms)
                if (j < E)
                    s_val[sb + q * (THREADS + THREADS / ITEMS)] =
                        ((uint32_t)c[q] < (uint64_t)ncol) ? (ident ? c[q] : __ldcg(gf + c[q])) : INF;
            }
        }
        __syncthreads();

        // phase 2: every thread walks ITEMS consecutive merge-path items
        // (row ends and entries) and min-reduces entries per row.  The walk
        // keeps the open row's end in a register; it reads an entry only while
        // y < that end <= E (or, for the row still open at the tile end, while
        // items remain), so y stays inside the tile.
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
                    if (acc != INF) atomicMin(&s_mngf[r], acc);
                    acc = INF;
                    ++r;
                    rend = r < nfull ? s_rowend[r] : 0x7fffffff;
                } else {
                    acc = min(acc, s_val[stage_at<ITEMS>(y)]);
                    ++y;
                }
            }
        }
        // the row still open at the end of each thread's items: when a whole
        // warp ends inside one row (a hub), reduce in registers first
        {
            const int key = (acc != INF && r >= 0 && r < R) ? r : -1;
            const int key0 = __shfl_sync(0xffffffffu, key, 0);
            if (__all_sync(0xffffffffu, key == key0)) {
                const int32_t wmin = (int32_t)__reduce_min_sync(0xffffffffu, (unsigned)acc);
                if ((tid & 31) == 0 && key0 >= 0) atomicMin(&s_mngf[key0], wmin);
            } else if (key >= 0) {
                atomicMin(&s_mngf[key], acc);
            }
        }
        __syncthreads();

        // phase 3: the tile's row minima into mngf.  A row that starts and
        // ends inside this tile has its complete minimum here: a plain store.
        // Only the first and last row of a tile can continue in a
        // neighbouring tile; those merge by atomic min.  (Atomic merges of
        // every row measured 2.6x slower on this kernel.)  A column block's
        // runs all merge by atomic min without a return value.
        if (!merge) {
            const bool first_whole = rp_at(rp, x0) >= y0;
            for (int i = tid; i < R; i += THREADS) {
                const int32_t mn = s_mngf[i];
                if (i < nfull && (i > 0 || first_whole))
                    mngf[x0 + i] = mn;
                else if (mn != INF)
                    atomicMin(mngf + x0 + i, mn);
            }
        } else {
            const int32_t* __restrict__ rowmap = S->rowmap + x0;
            for (int i = tid; i < R; i += THREADS) {
                const int32_t mn = s_mngf[i];
                if (mn == INF) continue;
                const int32_t u = rowmap[i] & 0x7fffffff;
                if (u < ncol) atomicMin(mngf + u, mn);
            }
        }
        __syncthreads();
    }
}

template <int THREADS, int ITEMS>
constexpr int k2_smem_bytes() {
    return (2 * (THREADS * ITEMS + 1) + THREADS * ITEMS + THREADS) * (int)sizeof(int32_t);
}

// a1 in the first iteration of a column-blocked solve, on the graph's own
// CSR (segment 0, its merge-path tiles of FIRST_THREADS x FIRST_ITEMS
// items): gf is still the identity (Algorithm 2 starts from f[u] = u), so
// mngf[u] is u's smallest neighbour id and nothing is gathered.  The same
// walk counts, per tile and column block, the tile's entries and runs (see
// the block copy's layout) into cnt[b][t] and cnt[nb + b][t] (rows of
// tiles + 1 entries, the last one 0; a chunk's exclusive scan over its tiles
// turns them into offsets, and its sum is the chunk's total): every thread
// follows its items' segments of one row and one block and adds each
// segment to the tile's counters when it ends.
constexpr int FIRST_THREADS = 64;
constexpr int FIRST_ITEMS = 16;
static_assert(FIRST_THREADS * FIRST_ITEMS == BUILD_TILE, "the block copy cuts along the first iteration's tiles");
static_assert(FIRST_THREADS >= 2 * MAX_COL_BLOCKS, "one thread per count of a tile");

template <typename RP>
__global__ void __launch_bounds__(FIRST_THREADS)
    k2_first(Ctx* __restrict__ ctx, int32_t* __restrict__ cnt, int nb, int shift, const int64_t* __restrict__ range,
             int chunk) {
    constexpr int THREADS = FIRST_THREADS, ITEMS = FIRST_ITEMS, TILE = THREADS * ITEMS;
    extern __shared__ int32_t smem[];
    int32_t* s_rowend = smem;                // local end offset of each row in the tile
    int32_t* s_mngf = smem + (TILE + 1);     // per-row minimum over the tile's entries
    int32_t* s_col = smem + 2 * (TILE + 1);  // the tile's column ids as given (at stage_at)
    __shared__ int s_cnt[2 * MAX_COL_BLOCKS];
    const int tid = threadIdx.x;
    const Seg* __restrict__ S = ctx->segs;
    const RP* __restrict__ rp = (const RP*)S->rp;
    int32_t* mngf = S->mngf;
    const int64_t n = S->n, m = S->m;
    const bool count = cnt != nullptr;
    const int64_t T1 = (int64_t)S->k2_ntiles + 1;
    // range (may be null): this launch takes the tiles [range[chunk], range[chunk + 1])
    const int64_t lt0 = range ? range[chunk] : 0, lt1 = range ? range[chunk + 1] : S->k2_ntiles;
    if (count && blockIdx.x == 0 && chunk == 0 && tid < 2 * nb) cnt[(int64_t)tid * T1 + T1 - 1] = 0;
    if (tid < 2 * MAX_COL_BLOCKS) s_cnt[tid] = 0;
    __syncthreads();
    for (int64_t lt = lt0 + blockIdx.x; lt < lt1; lt += gridDim.x) {
        const int64_t t = S->k2_tile0 + lt;
        const int64_t d0 = lt * TILE;
        const int64_t d1 = min(d0 + (int64_t)TILE, n + m);
        const int64_t x0 = ctx->k2_tile_row[t];
        const int64_t x1 = (lt + 1 < S->k2_ntiles) ? (int64_t)ctx->k2_tile_row[t + 1] : n;
        if (x1 < x0 || x1 - x0 > d1 - d0) {  // only possible for a malformed row_ptr
            if (count && tid < 2 * nb) cnt[(int64_t)tid * T1 + lt] = 0;
            continue;
        }
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
            s_mngf[i] = INF;
        }
        {
            int32_t c[ITEMS];
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const int j = tid + q * THREADS;
                c[q] = j < E ? ld_stream(cit + j) : 0;
            }
            const int sb = stage_at<ITEMS>(tid);
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const int j = tid + q * THREADS;
                if (j < E) s_col[sb + q * (THREADS + THREADS / ITEMS)] = c[q];
            }
        }
        __syncthreads();

        // the merge-path walk of k2_spmv over ITEMS items per thread, and the
        // thread's segments (consecutive entries of one row in one block):
        // a segment starts a run unless it continues the run of the entry
        // before it (same row, same block)
        const int k0 = tid * ITEMS;
        int r = -1;
        int32_t acc = INF;
        int cb = -1, clen = 0;
        bool cstart = false;
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
                    if (acc != INF) atomicMin(&s_mngf[r], acc);
                    acc = INF;
                    if (count && clen) {
                        atomicAdd(&s_cnt[cb], clen);
                        if (cstart) atomicAdd(&s_cnt[MAX_COL_BLOCKS + cb], 1);
                    }
                    cb = -1;
                    clen = 0;
                    ++r;
                    rend = r < nfull ? s_rowend[r] : 0x7fffffff;
                } else {
                    const int32_t v = s_col[stage_at<ITEMS>(y)];
                    if ((uint32_t)v < (uint64_t)n) acc = min(acc, v);
                    if (count) {
                        const int b = col_block(v, shift, nb);
                        if (b != cb) {
                            if (clen) {
                                atomicAdd(&s_cnt[cb], clen);
                                if (cstart) atomicAdd(&s_cnt[MAX_COL_BLOCKS + cb], 1);
                            }
                            // a new segment inside the thread's items of one row
                            // always starts a run; the thread's first segment of
                            // a row does unless the entry before it (same row)
                            // has the same block
                            const int rs = r > 0 ? s_rowend[r - 1] : 0;
                            cstart = cb >= 0 || y == 0 || (r > 0 && y == rs) ||
                                     col_block(s_col[stage_at<ITEMS>(y - 1)], shift, nb) != b;
                            cb = b;
                            clen = 0;
                        }
                        ++clen;
                    }
                    ++y;
                }
            }
        }
        if (count && clen) {
            atomicAdd(&s_cnt[cb], clen);
            if (cstart) atomicAdd(&s_cnt[MAX_COL_BLOCKS + cb], 1);
        }
        {
            const int key = (acc != INF && r >= 0 && r < R) ? r : -1;
            const int key0 = __shfl_sync(0xffffffffu, key, 0);
            if (__all_sync(0xffffffffu, key == key0)) {
                const int32_t wmin = (int32_t)__reduce_min_sync(0xffffffffu, (unsigned)acc);
                if ((tid & 31) == 0 && key0 >= 0) atomicMin(&s_mngf[key0], wmin);
            } else if (key >= 0) {
                atomicMin(&s_mngf[key], acc);
            }
        }
        __syncthreads();

        // row minima into mngf: rows whole in the tile by plain stores, the
        // first and last row (they may continue in a neighbouring tile) by
        // atomic min
        const bool first_whole = rp_at(rp, x0) >= y0;
        for (int i = tid; i < R; i += THREADS) {
            const int32_t mn = s_mngf[i];
            if (i < nfull && (i > 0 || first_whole))
                mngf[x0 + i] = mn;
            else if (mn != INF)
                atomicMin(mngf + x0 + i, mn);
        }
        if (count) {
            if (tid < nb)
                cnt[(int64_t)tid * T1 + lt] = s_cnt[tid];
            else if (tid >= MAX_COL_BLOCKS && tid < MAX_COL_BLOCKS + nb)
                cnt[(int64_t)(nb + tid - MAX_COL_BLOCKS) * T1 + lt] = s_cnt[tid];
        }
        __syncthreads();
        if (tid < 2 * MAX_COL_BLOCKS) s_cnt[tid] = 0;
        __syncthreads();
    }
}

// Entry bounds of the chunks in which col_idx arrives from host memory, and
// for each bound the number of first-iteration tiles whose entries all lie
// below it (tiles end at non-decreasing entry positions, so each count is a
// binary search): chunk c's launch of k2_first takes tiles [out[c], out[c+1]).
struct FeedBounds {
    int64_t b[MAX_FEED_CHUNKS + 1];  // b[c + 1]: entries copied once chunk c has landed
    int32_t chunks;
};

__global__ void k_feed_tiles(const Ctx* __restrict__ ctx, FeedBounds fb, int64_t* __restrict__ out) {
    const Seg& S = ctx->segs[0];
    const int64_t T = S.k2_ntiles, n = S.n, m = S.m, tile = ctx->k2_tile;
    const int32_t* tile_row = ctx->k2_tile_row + S.k2_tile0;
    const int c = threadIdx.x;
    if (c > fb.chunks) return;
    if (c == 0 || c == fb.chunks) {
        out[c] = c == 0 ? 0 : T;
        return;
    }
    // tiles t < lo end at or below the bound: y1(t) = min((t + 1) tile, n + m) - x1(t)
    const int64_t bound = fb.b[c];
    int64_t lo = 0, hi = T;
    while (lo < hi) {
        const int64_t t = (lo + hi) >> 1;
        const int64_t d1 = min((t + 1) * tile, n + m);
        const int64_t x1 = t + 1 < T ? (int64_t)tile_row[t + 1] : n;
        if (d1 - x1 <= bound)
            lo = t + 1;
        else
            hi = t;
    }
    out[c] = lo;
}

__host__ __device__ constexpr int k2_first_smem() {
    return (3 * (FIRST_THREADS * FIRST_ITEMS) + 2 + FIRST_THREADS) * (int)sizeof(int32_t);
}

// a1, sparse iteration (Section 4.2's SpMSpV): only vertices whose gf
// changed in the last iteration can lower a neighbour's minimum, and gf never
// increases, so min(old mngf, pushes of the new gf of changed vertices) is
// exactly the SpMV of the new gf.  One warp per changed vertex; each graph
// decides for itself, after every iteration, whether it pushes or runs a
// full SpMV, and the frontier holds (graph, vertex) pairs of all of them.
template <typename RP>
__global__ void __launch_bounds__(256) k2_push(Ctx* __restrict__ ctx) {
    if (!(ctx->mode & MODE_PUSH)) return;
    const Seg* __restrict__ segs = ctx->segs;
    if (blockIdx.x == 0 && threadIdx.x == 0 && segs[0].active && segs[0].mode == 1) ctx->sparse_iters++;
    const int32_t* __restrict__ F = ctx->frontier;
    const unsigned len = ctx->frontier_len;
    const int nsegs = ctx->num_segs;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < len; i += nwarps) {
        const int32_t sg = F[2 * i], v = F[2 * i + 1];
        if ((uint32_t)sg >= (uint32_t)nsegs) continue;
        const Seg& S = segs[sg];
        if (!S.active || S.mode != 1 || (uint32_t)v >= (uint64_t)S.n) continue;
        const RP* rp = (const RP*)S.rp;
        const int32_t g = S.gf[v];
        int64_t b = rp_at(rp, v), e = rp_at(rp, v + 1);
        if (b < 0) b = 0;
        if (e > S.m) e = S.m;
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t u = S.ci[k];
            if ((uint32_t)u < (uint64_t)S.n) atomicMin(S.mngf + u, g);
        }
    }
}

// a2 + a3: hooks from mngf for every vertex of every active graph.
//   stochastic hooking  f_next[f[u]] <-min mngf[u]  (a no-op unless mngf[u] <
//                        gf[u], because f[p[u]] <= p[p[u]] = gf[u] throughout)
//   aggressive hooking  f_next[u] <-min mngf[u]
//   shortcutting        f_next[u] <-min gf[u]
// Many vertices hook to the same root (the hot spot of Section 4.2): a
// stochastic hook first reads the root's current value and issues its atomic
// only when it would lower it.  f only decreases, so a skipped atomic could
// not have changed it, and the result is the same minimum.
__global__ void __launch_bounds__(K3_THREADS) k2_hook(Ctx* __restrict__ ctx) {
    const int64_t T = ctx->k3_total;
    const int tid = threadIdx.x;
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        const Seg* S = ctx->segs + ctx->k3_tile_seg[t];
        if (!S->active) continue;
        const int64_t n = S->n;
        const int64_t v0 = (t - S->k3_tile0) * K3_TILE;
        const int32_t* __restrict__ mngf = S->mngf;
        const int32_t* __restrict__ gf = S->gf;
        const int32_t* __restrict__ p = S->p;
        int32_t* f = S->f;
        int32_t mn[K3_ITEMS], g[K3_ITEMS], pu[K3_ITEMS];
#pragma unroll
        for (int q = 0; q < K3_ITEMS; ++q) {
            const int64_t v = v0 + tid + q * K3_THREADS;
            mn[q] = v < n ? mngf[v] : INF;
        }
#pragma unroll
        for (int q = 0; q < K3_ITEMS; ++q) {
            const int64_t v = v0 + tid + q * K3_THREADS;
            const bool live = mn[q] != INF;
            g[q] = live ? gf[v] : 0;
            pu[q] = live ? p[v] : 0;
        }
#pragma unroll
        for (int q = 0; q < K3_ITEMS; ++q) {
            if (mn[q] == INF) continue;
            const int64_t v = v0 + tid + q * K3_THREADS;
            if (mn[q] < g[q] && mn[q] < __ldcg(f + pu[q])) atomicMin(f + pu[q], mn[q]);
            const int32_t m2 = mn[q] < g[q] ? mn[q] : g[q];
            if (m2 < pu[q]) atomicMin(f + v, m2);
        }
    }
}

// ---------------------------------------------------------------------------
// K3: grandparents, termination count, snapshot; last CTA closes the iteration
// ---------------------------------------------------------------------------

__device__ __forceinline__ void close_iteration(Ctx* ctx, cudaGraphConditionalHandle cond, int use_cond) {
    const int tid = threadIdx.x;
    const int G = ctx->num_segs;
    const int max_iters = ctx->max_iters;
    const bool sparse = ctx->sparse_enabled && !ctx->frontier_overflow;
    const int div = ctx->sparse_div > 0 ? ctx->sparse_div : 1;
    int any = 0, dense = 0, push = 0;
    for (int s = tid; s < G; s += blockDim.x) {
        Seg* S = ctx->segs + s;
        if (!S->active || S->leader != s) continue;  // column blocks follow their graph
        unsigned int ch = atomicExch(&S->changed, 0u);
        const unsigned long long deg = S->fr_deg;
        S->fr_deg = 0;
        int it = S->iters + 1;
        S->iters = it;
        if (s == 0 && it <= TRACE_LEN) ctx->sum.trace[it - 1] = ch;
        if (ch == 0) {
            S->active = 0;
            S->converged = 1;
        } else if (it >= max_iters) {
            S->active = 0;
            S->status |= DEV_ERR_MAX_ITERS;
        } else {
            any = 1;
            // next iteration: push from the vertices whose gf just changed
            // when their rows are few enough, else a full SpMV
            S->mode = (sparse && deg <= (unsigned long long)(S->m / div)) ? 1 : 0;
            if (S->mode)
                push = 1;
            else
                dense = 1;
        }
    }
    any = __syncthreads_or(any);
    dense = __syncthreads_or(dense);
    push = __syncthreads_or(push);
    if (tid == 0) {
        ctx->k3_done = 0;
        int li = ctx->loop_iter + 1;
        ctx->loop_iter = li;
        ctx->any_active = any;
        ctx->frontier_len = ctx->frontier_next;
        ctx->frontier_next = 0;
        ctx->frontier_overflow = 0;
        ctx->mode = (dense ? MODE_DENSE : 0) | (push ? MODE_PUSH : 0);
        if (use_cond) cudaGraphSetConditional(cond, (any && li < ctx->loop_limit) ? 1u : 0u);
    }
}

template <typename RP>
__global__ void __launch_bounds__(K3_THREADS)
    k3_grandparent(Ctx* __restrict__ ctx, cudaGraphConditionalHandle cond, int use_cond) {
    __shared__ int s_red[K3_THREADS / 32];
    __shared__ int s_woff[K3_THREADS / 32];
    __shared__ unsigned s_base;
    __shared__ int s_last;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int64_t T = ctx->k3_total;
    const bool track = ctx->sparse_enabled != 0;
    for (int64_t t = blockIdx.x; t < T; t += gridDim.x) {
        Seg* S = ctx->segs + ctx->k3_tile_seg[t];
        if (!S->active) continue;
        const int64_t n = S->n;
        const int64_t v0 = (t - S->k3_tile0) * K3_TILE;
        int32_t* f = S->f;
        int32_t* p = S->p;
        int32_t* gf = S->gf;
        // all loads of a thread first (f[v], gf[v], then the gathers f[f[v]])
        int32_t fu[K3_ITEMS], old[K3_ITEMS], g[K3_ITEMS];
#pragma unroll
        for (int q = 0; q < K3_ITEMS; ++q) {
            const int64_t v = v0 + tid + q * K3_THREADS;
            fu[q] = v < n ? f[v] : 0;
            old[q] = v < n ? gf[v] : 0;
        }
#pragma unroll
        for (int q = 0; q < K3_ITEMS; ++q) g[q] = f[fu[q]];
        int c = 0;
        unsigned masks[K3_ITEMS];
#pragma unroll
        for (int q = 0; q < K3_ITEMS; ++q) {
            const int64_t v = v0 + tid + q * K3_THREADS;
            const bool ch = v < n && g[q] != old[q];
            if (v < n) {
                if (ch) {
                    gf[v] = g[q];
                    ++c;
                }
                p[v] = fu[q];
            }
            masks[q] = __ballot_sync(0xffffffffu, ch);
        }
        c = __reduce_add_sync(0xffffffffu, c);  // == popcounts of the masks, summed
        if (lane == 0) s_red[tid >> 5] = c;
        __syncthreads();
        if (tid == 0) {
            // one reservation per tile in the next iteration's frontier
            int total = 0;
            for (int w = 0; w < K3_THREADS / 32; ++w) {
                const int x = s_red[w];
                s_woff[w] = total;
                total += x;
            }
            if (total) atomicAdd(&S->changed, (unsigned int)total);
            s_base = 0xffffffffu;  // no room: the frontier is dropped for one iteration
            if (track && total) {
                const unsigned b = atomicAdd(&ctx->frontier_next, (unsigned)total);
                if ((unsigned long long)b + total <= ctx->frontier_cap)
                    s_base = b;
                else
                    ctx->frontier_overflow = 1;
            }
        }
        __syncthreads();
        if (track && c) {
            // frontier of the next iteration: the (graph, vertex) pairs of
            // this tile's changed vertices, and the sum of their degrees
            const int32_t sg = ctx->k3_tile_seg[t];
            const RP* rp = (const RP*)S->rp;
            const bool room = s_base != 0xffffffffu;
            unsigned off = s_base + (unsigned)s_woff[tid >> 5];
            unsigned long long dsum = 0;
#pragma unroll
            for (int q = 0; q < K3_ITEMS; ++q) {
                const unsigned mask = masks[q];
                if (mask >> lane & 1u) {
                    const int64_t v = v0 + tid + q * K3_THREADS;
                    if (room) {
                        const int64_t at = 2 * (int64_t)(off + __popc(mask & ((1u << lane) - 1u)));
                        ctx->frontier[at] = sg;
                        ctx->frontier[at + 1] = (int32_t)v;
                    }
                    dsum += (unsigned long long)(rp_at(rp, v + 1) - rp_at(rp, v));
                }
                off += (unsigned)__popc(mask);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
            if (lane == 0 && dsum) atomicAdd(&S->fr_deg, dsum);
        }
        __syncthreads();
    }
    // the last CTA to arrive closes the iteration for every segment
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        unsigned int ticket = atomicAdd(&ctx->k3_done, 1u);
        s_last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    close_iteration(ctx, cond, use_cond);
}

// end of a call: per-graph iteration counts and the summary
// per-call summary; also counts the call's device-loop kernels (loop_iter
// iterations of loop_kernels each) into the context's running total
__global__ void k_finish(Ctx* ctx, int32_t* iters_out, int loop_kernels) {
    __shared__ long long s_it[256];
    __shared__ int s_st[256], s_cv[256], s_act[256];
    const int G = ctx->num_segs;
    long long it = 0;
    int st = 0, cv = 1, act = 0;
    for (int s = threadIdx.x; s < G; s += blockDim.x) {
        const Seg& S = ctx->segs[s];
        if (S.leader != s) continue;  // column blocks carry no state of their own
        if (iters_out) iters_out[s] = S.iters;
        it = max(it, (long long)S.iters);
        st |= S.status;
        cv &= S.converged;
        act += S.active;
    }
    s_it[threadIdx.x] = it;
    s_st[threadIdx.x] = st;
    s_cv[threadIdx.x] = cv;
    s_act[threadIdx.x] = act;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s_it[threadIdx.x] = max(s_it[threadIdx.x], s_it[threadIdx.x + off]);
            s_st[threadIdx.x] |= s_st[threadIdx.x + off];
            s_cv[threadIdx.x] &= s_cv[threadIdx.x + off];
            s_act[threadIdx.x] += s_act[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctx->sum.iterations = s_it[0];
        ctx->sum.status = s_st[0] | ctx->val_status;
        ctx->sum.converged = s_cv[0];
        ctx->sum.loop_iter = ctx->loop_iter;
        ctx->sum.num_active = s_act[0];
        ctx->sum.sparse_iters = ctx->sparse_iters;
        ctx->loop_kernels_total += (unsigned long long)ctx->loop_iter * (unsigned long long)loop_kernels;
        ctx->sum.loop_kernels = ctx->loop_kernels_total;
    }
}

}  // namespace fsv

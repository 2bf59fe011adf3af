// fastsv_types.cuh -- device data structures shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fsv {

constexpr int32_t INF = 0x7fffffff;
constexpr int K3_THREADS = 256;
constexpr int K3_ITEMS = 8;
constexpr int K3_TILE = K3_THREADS * K3_ITEMS;
constexpr int TRACE_LEN = 64;

// status bits written by device code
constexpr int32_t DEV_ERR_MAX_ITERS = 1;
constexpr int32_t DEV_ERR_BAD_ROWPTR = 2;
constexpr int32_t DEV_ERR_BAD_COLIDX = 4;
constexpr int32_t DEV_ERR_ASYMMETRIC = 8;

struct Seg {
    const void* rp;      // row pointers (int32 or int64 by kernel instance), n+1 entries, local offsets
    const int32_t* ci;   // neighbour ids (local)
    int32_t* f;          // parent vector (caller's labels buffer)
    int32_t* p;          // snapshot of f
    int32_t* gf;         // grandparents
    int64_t n, m;
    int64_t k2_tile0;    // first hooking tile of this segment in the global list
    int64_t k3_tile0;    // first grandparent tile
    int32_t k2_ntiles, k3_ntiles;
    int32_t active;      // 1 while iterating
    int32_t iters;       // iterations executed
    int32_t status;      // DEV_ERR_* bits
    int32_t converged;   // 1 once an iteration left gf unchanged
    unsigned int changed;  // this iteration's changed-grandparent count
    int32_t user;        // owner tag (pool slot id), unused by the kernels
    int32_t leader;      // segment whose state governs this one: itself, or for a
                         // column block of a graph, the graph's own segment
    int32_t mode;        // this iteration: 0 = full SpMV, 1 = push from the frontier
    int32_t* mngf;       // per-row minimum of gf over neighbours, kept across iterations
    unsigned long long fr_deg;  // degree sum of this iteration's changed vertices (being filled)
    const int32_t* rowmap;  // column block of a graph: the graph row of each local row (a run of
                            // entries; bit 31 set: merge its minimum atomically); nullptr: identity
};

constexpr int MAX_COL_BLOCKS = 32;   // column blocks of one graph
constexpr int MAX_FEED_CHUNKS = 16;  // chunks of the column-block copy (and of a host-fed col_idx)

// where the blocks of one chunk of the column-block copy start in colB and
// rowsB (computed on the device from the chunk's scanned totals; entry b + 1
// is the end of block b)
struct ChunkLayout {
    int64_t ebase[MAX_COL_BLOCKS + 1];
    int64_t pbase[MAX_COL_BLOCKS + 1];
};

// Ctx::mode bits: some active graph runs a full SpMV / pushes this iteration
constexpr int32_t MODE_DENSE = 1;
constexpr int32_t MODE_PUSH = 2;

struct Summary {
    int64_t iterations;     // max over segments
    int32_t status;         // OR over segments and validation
    int32_t converged;      // AND over segments
    int32_t loop_iter;      // iterations the device loop executed in this call
    int32_t num_active;     // segments still active
    int32_t sparse_iters;   // iterations that pushed from the frontier instead of a full SpMV
    int32_t pad;
    unsigned long long loop_kernels;  // device-loop kernel launches of every call on this context so far
    unsigned long long trace[TRACE_LEN];  // segment 0: changed count per iteration
};

struct Ctx {
    Seg* segs;
    int32_t num_segs;
    int32_t k2_tile;         // merge-path items per hooking tile
    int64_t k2_total;        // hooking tiles over all segments
    int64_t k3_total;        // grandparent tiles over all segments
    int32_t* k2_tile_seg;
    int32_t* k2_tile_row;    // merge-path start row of each hooking tile (segment-local)
    int32_t* k3_tile_seg;
    int32_t max_iters;
    int32_t loop_limit;      // iterations allowed in this launch of the device loop
    int32_t loop_iter;       // iterations executed in this launch
    unsigned int k3_done;    // CTA ticket for the last-block epilogue
    int32_t any_active;
    int32_t val_status;      // validation result bits
    // sparse iterations: a graph whose changed vertices have a degree sum of at
    // most m / sparse_div pushes their new gf to the neighbours' mngf instead
    // of running a full SpMV (decided per graph after every iteration)
    int32_t sparse_enabled;
    int32_t mode;                  // MODE_DENSE | MODE_PUSH: the kinds of work this iteration has
    int32_t* frontier;             // (segment, vertex) pairs whose gf changed in the last iteration
    unsigned int frontier_len;     // pairs in the frontier
    unsigned int frontier_next;    // being filled by this iteration's k3
    unsigned int frontier_cap;     // pairs the buffer holds
    int32_t frontier_overflow;     // this iteration's changes did not fit: no pushes next
    int32_t sparse_div;
    int32_t sparse_iters;          // iterations graph 0 ran in push mode in this call
    unsigned long long loop_kernels_total;  // device-loop kernel launches over all calls (never reset)
    int32_t blk_chunks;            // segments per column block of graph 0 (one per chunk of its copy)
    Summary sum;
};

}  // namespace fsv

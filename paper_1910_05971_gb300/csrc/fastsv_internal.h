// fastsv_internal.h -- host-side handle shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/fastsv.h"
#include "fastsv_types.cuh"

namespace fsv {

struct GraphKey {
    int rp64;
    int items;
    int mode;
    const void* ctx;
    bool operator<(const GraphKey& o) const {
        if (rp64 != o.rp64) return rp64 < o.rp64;
        if (items != o.items) return items < o.items;
        if (mode != o.mode) return mode < o.mode;
        return ctx < o.ctx;
    }
};

struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
};

struct Pool;  // serving pool (pool.cu)

// one line of the tuning cache (tune.cu)
struct TuneEntry {
    std::string key;
    int32_t k2_items, k2_threads, col_blocks, sparse_div, batch_sparse_div;
};
enum { TUNE_SINGLE = 0, TUNE_BATCHED = 1 };

}  // namespace fsv

struct fastsv_ctx {
    fastsv_options opt;        // options of the current call (base_opt, or with a tuning-cache entry applied)
    fastsv_options base_opt;   // options the handle was created with
    std::vector<fsv::TuneEntry> tune;
    int32_t last_tuned = 0;
    int device = 0;
    int num_sms = 0;
    int64_t l2_bytes = 0;
    cudaStream_t last_stream = nullptr;

    // device context and workspace
    fsv::Ctx* d_ctx = nullptr;
    fsv::Seg* d_segs = nullptr;
    int64_t cap_segs = 0;
    int32_t* d_k2_seg = nullptr;
    int32_t* d_k2_row = nullptr;
    int64_t cap_k2 = 0;
    int32_t* d_k3_seg = nullptr;
    int64_t cap_k3 = 0;
    int32_t* d_p = nullptr;
    int32_t* d_gf = nullptr;
    int32_t* d_mngf = nullptr;       // per-row neighbour minimum, kept across iterations
    int32_t* d_frontier = nullptr;   // vertices whose gf changed in the last iteration
    int64_t cap_n = 0;

    // column-blocked copy of a large graph (see k_block_split)
    int32_t* d_counts = nullptr;    // per (block, tile) entries and runs, scanned in place per chunk
    int64_t cap_blk = 0;
    int32_t* d_sums = nullptr;
    int64_t cap_sums = 0;
    int32_t* d_colB = nullptr;      // the entries, chunk after chunk, in a chunk block after block
    int64_t cap_colB = 0;
    int32_t* d_rowsB = nullptr;     // graph row of every run
    int32_t* d_endsB = nullptr;     // end of every run inside its (chunk, block) (one leading 0 each)
    int64_t cap_runs = 0;
    fsv::ChunkLayout* d_clay = nullptr;  // per chunk: where its blocks start
    int32_t* d_ctot = nullptr;           // per chunk: entries and runs of each block
    int64_t* d_build_scalars = nullptr;  // the copy's totals and consistency for the host
    int64_t last_runs = 0;
    int last_col_blocks = 1;

    // the host-buffer entry point's copy of col_idx in chunks, overlapping the
    // first iteration of a column-blocked solve
    cudaStream_t feed_stream = nullptr;
    cudaEvent_t feed_ev[17] = {};        // [0]: the call's stream reached the copies; [1 + c]: chunk c landed
    // a column-blocked graph's first hooks run beside its block copy
    cudaStream_t side_stream = nullptr;
    cudaEvent_t side_ev[2] = {};         // [0]: the first iteration's SpMV is done; [1]: its hooks are
    int64_t* d_feed_tiles = nullptr;     // first-iteration tile range of every chunk

    // device copies for the host-buffer entry point
    void* d_rp_copy = nullptr;
    size_t cap_rp_copy = 0;
    int32_t* d_ci_copy = nullptr;
    size_t cap_ci_copy = 0;
    int32_t* d_lab_copy = nullptr;
    size_t cap_lab_copy = 0;

    // pinned host staging
    fsv::Summary* h_sum = nullptr;
    int64_t* h_scalar = nullptr;

    cudaEvent_t ev_start = nullptr, ev_setup = nullptr, ev_end = nullptr;
    bool have_timing = false;

    std::map<fsv::GraphKey, fsv::LoopGraph> graphs;
    int k2_grid = 0, k3_grid = 0;

    // bookkeeping of the last call
    int64_t last_n = 0, last_m = 0;
    int last_status = 0;
    int last_cuda_error = 0;
    bool pending = false;      // a call whose summary has not been read yet
    bool single = true;        // last call was a single-graph call
    float ms_k2 = 0.f, ms_k3 = 0.f, ms_push = 0.f, ms_hook = 0.f;
    int32_t dense_iters = 0;   // host loop: timed iterations that ran the full SpMV
    int32_t timed_iters = 0;   // host loop: iterations timed by ms_k2 .. ms_hook
    float ms_total_cache = 0.f, ms_setup_cache = 0.f;
    int64_t launches = 0;      // kernels launched, settled by fastsv_get_stats
    int64_t pending_fixed_launches = 0;  // set-up kernels of the pending call
    int64_t launches_loop_dev = 0;       // device-loop kernels of every call up to the last synchronised one
    int pending_loop_kernels = 0;        // kernels per device-loop iteration of the pending call
    int alloc_count = 0;
    int32_t loop_limit_host = 0;         // iteration cap of the host-loop mode
    bool pool_loop_pending = false;      // a pool step's device loop whose kernels are not counted yet

    fsv::Pool* pool = nullptr;
};

namespace fsv {

// error plumbing
fastsv_status cuda_fail(fastsv_ctx* h, cudaError_t e);
#define FSV_CUDA(h, call)                                  \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return fsv::cuda_fail(h, _e); \
    } while (0)

// device allocation through the handle (counts allocations for the test hook)
fastsv_status dev_alloc(fastsv_ctx* h, void** p, size_t bytes);
fastsv_status ensure_workspace(fastsv_ctx* h, int64_t n, int64_t k2_tiles, int64_t k3_tiles, int64_t segs);
fastsv_status get_loop_graph(fastsv_ctx* h, Ctx* ctx, int rp64_orig, int rp64_dense, int items, int nblocks,
                             LoopGraph** out);
fastsv_status run_loop(fastsv_ctx* h, Ctx* ctx, int rp64_orig, int rp64_dense, int items, int nblocks,
                       cudaStream_t s);
fastsv_status rebuild_tiles(fastsv_ctx* h, Ctx* ctx, cudaStream_t s);
int setup_grid(const fastsv_ctx* h);
int k2_items(const fastsv_ctx* h);
int k2_threads(const fastsv_ctx* h);
int64_t k2_tile(const fastsv_ctx* h);
void pool_release(fastsv_ctx* h);
int tune_key(int kind, int64_t n, int64_t m, int64_t graphs, int bits, char* out, size_t cap);
fastsv_status tune_load(fastsv_ctx* h, const char* path);
void tune_apply(fastsv_ctx* h, int kind, int64_t n, int64_t m, int64_t graphs, int bits);

}  // namespace fsv

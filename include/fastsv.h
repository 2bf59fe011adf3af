/*
 * fastsv.h -- C ABI of libfastsv, FastSV connected components on one GB300 GPU.
 *
 * Method: Y. Zhang, A. Azad, Z. Hu, "FastSV: A Distributed-Memory Connected
 * Component Algorithm with Fast Convergence" (arXiv:1910.05971).
 *
 * Every solve runs Algorithm 2 (Section 3) on the device:
 *   repeat
 *     mngf[u]      = min_{v in N(u)} gf[v]          ((select2nd,min) SpMV, Section 4.1)
 *     f_next[f[u]] <-min mngf[u]                    stochastic hooking (Section 3.2)
 *     f_next[u]    <-min mngf[u]                    aggressive hooking (Section 3.3)
 *     f_next[u]    <-min gf[u]                      shortcutting
 *     f <- f_next;  gf <- f[f]
 *   until gf is unchanged                            early termination (Section 3.4)
 * and returns labels[u] = f[u] = the smallest vertex id in u's connected
 * component (the converged state of Section 3.4, proved in Appendix A).
 * All arithmetic is int32 compare/min; results are exact and deterministic.
 *
 * Conventions for every entry point:
 *  - Graphs are undirected and given in CSR form with each edge {u,v} stored
 *    in both rows (symmetric).  Self-loops and duplicate entries are allowed
 *    and change neither the labels nor the iteration sequence.  Rows need not
 *    be sorted.  Vertex ids are int32 in [0, n).
 *  - "device" pointers must point to memory of the current CUDA device;
 *    "host" pointers to host memory (pinned memory gives full copy speed).
 *    All arrays are owned by the caller; the library never frees them and
 *    keeps no reference after the call's work has completed on the stream.
 *  - The handle owns its device workspace (snapshot and grandparent vectors,
 *    tile lists, counters) and grows it on demand; it is freed by
 *    fastsv_destroy.  A handle is not thread-safe: use one per host thread.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; calls return after enqueueing, except
 *    where a call says it synchronises.
 *  - Argument errors detectable on the host return at once with
 *    FASTSV_ERR_INVALID_ARG and enqueue nothing.  Errors found on the device
 *    (iteration cap, invalid CSR when validation is on) are reported by
 *    fastsv_get_stats.
 */
#ifndef FASTSV_H
#define FASTSV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fastsv_ctx* fastsv_t;

typedef enum {
    FASTSV_OK = 0,
    FASTSV_ERR_INVALID_ARG = 1,   /* bad pointer, size or option; nothing was enqueued */
    FASTSV_ERR_OOM = 2,           /* device or pinned allocation failed; the handle stays usable */
    FASTSV_ERR_CUDA = 3,          /* a CUDA runtime call failed; see fastsv_last_cuda_error */
    FASTSV_ERR_MAX_ITERS = 4,     /* the iteration cap was reached before f[f] stopped changing */
    FASTSV_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    FASTSV_ERR_UNSUPPORTED = 6,   /* option or size this build does not handle */
    FASTSV_ERR_INVALID_GRAPH = 7, /* validation found a malformed CSR (bounds, monotonicity, symmetry) */
    FASTSV_ERR_FULL = 8           /* pool: no slot or not enough budget for the request right now */
} fastsv_status;

/* Solver modes.  FASTSV_MODE_SYNC is Algorithm 2 exactly: every update of
 * an iteration reads the vectors as they were at its start (the f / f_next
 * separation of Section 2.4), so the pointer graph after iteration i is the
 * same on every run and equal to the CPU oracle's.  FASTSV_MODE_ASYNC reads
 * and writes one parent vector in place (the concurrent variant Section 2.4
 * mentions): one fused kernel per iteration hooks f[f[u]] and f[u] onto the
 * row minimum of the live f[v] and shortcuts f[u] to f[f[u]]; the loop stops
 * after an iteration that lowered no entry of f.  Labels are the same as in
 * FASTSV_MODE_SYNC; the iteration count and changed_per_iter (rows whose
 * processing lowered some entry) depend on the schedule.  Single-graph calls
 * only: fastsv_cc_batched and fastsv_pool_create return
 * FASTSV_ERR_UNSUPPORTED on an asynchronous handle. */
enum { FASTSV_MODE_SYNC = 0, FASTSV_MODE_ASYNC = 1 };

typedef struct {
    int32_t rowptr_bits;   /* width of row_ptr entries in fastsv_cc / fastsv_cc_host: 32 or 64 (default 64) */
    int32_t mode;          /* FASTSV_MODE_SYNC (default) or FASTSV_MODE_ASYNC */
    int32_t max_iters;     /* iteration cap per graph (default 4096); reaching it gives FASTSV_ERR_MAX_ITERS */
    int32_t validate;      /* 0 off (default); 1 check row_ptr monotonicity and neighbour ids in [0,n);
                              2 also check symmetry (rows must then be sorted).  Validation synchronises. */
    int32_t use_graph;     /* 1 (default): the iteration loop runs on the device inside a CUDA graph
                              conditional WHILE node, with no host synchronisation per iteration;
                              0: host loop, one synchronisation per iteration, per-kernel timings */
    int32_t k2_items;      /* merge-path items per thread in the hooking kernel (0 = default) */
    int32_t grid_ctas_per_sm; /* persistent CTAs per SM for the iteration kernels (0 = occupancy limit) */
    int32_t timing;        /* 1: record device time of each call with CUDA events (default 1) */
    int32_t fail_alloc_after; /* test hook: >0 makes the N-th workspace allocation of this handle fail
                                 (returns FASTSV_ERR_OOM); 0 off */
    int32_t col_blocks;    /* column blocks of the SpMV for one large graph: 0 = automatic (blocks when
                              4n bytes >= 1.5x the L2 and m >= 8n, one block per col_block_mib MiB of the
                              gathered vector), 1 = never, 2..32 = that many.  A blocked call copies
                              col_idx once into column-block order (needs m <= 2^31 - 1) and runs one
                              SpMV launch per block, whose gathers then hit an L2-resident slice of the
                              grandparent vector.  A block lists only the rows that have entries in it
                              (compressed rows).  Its first iteration runs before the copy, on the
                              caller's CSR (it gathers nothing), and counts the copy's sizes; the call
                              then synchronises once more, to size (or check) the copy's row lists (workspace:
                              4m bytes of entries, 8 bytes per (row, block) pair, 8nb bytes per 1024
                              entries of counts).  Rows need not be sorted (unsorted rows give longer
                              row lists and slower merges, never other labels) */
    int32_t k2_threads;    /* threads per CTA of the SpMV kernel: 256 (default) or 64 */
    int32_t sparse_div;    /* single-graph calls: an iteration pushes from the vertices whose grandparent
                              changed (SpMSpV, Section 4.2) instead of a full SpMV when the degree sum of
                              those vertices is at most m / sparse_div (default 2); 0 = always full SpMV */
    int32_t variant;       /* 0 (default) or 5: FastSV, Algorithm 2.  1..4: the convergence ablation of
                              Section 5.2 -- 1 = Algorithm 1 (simplified SV, Section 2.4), 2 = + hooking
                              to the grandparent (3.1), 3 = + stochastic hooking (3.2), 4 = Algorithm 2's
                              loop body with aggressive hooking (3.3) but stopping when f is unchanged
                              (no early termination, 3.4).  Variants 1..4 are deterministic per iteration,
                              run a host loop (one synchronisation per iteration), single-graph calls in
                              FASTSV_MODE_SYNC only; changed_per_iter then counts changed entries of f */
    int32_t batch_sparse_div; /* fastsv_cc_batched and pools: every graph decides after each iteration to
                              push from its changed vertices when their degree sum is at most
                              m_graph / batch_sparse_div; 0 (default) = always full SpMV.  Off by default:
                              on 4096 ER graphs the frontier bookkeeping cost more than the pushes saved
                              (139k graphs/s off, 116k at 4 to 32, 101k at 2) */
    int32_t col_block_mib; /* automatic column blocking (col_blocks = 0): MiB of the grandparent vector per
                              block (default 64, about half of the L2) */
    int32_t pool_wait_copies; /* pools: 0 (default) = a graph joins the first step after its copies to the
                              device have landed (copies overlap iterations); 1 = every step waits for the
                              copies of all graphs admitted before it, so a graph added before a step
                              always takes part in it */
    const char* tune_cache; /* NULL (default) or the path of a tuning cache written by the autotuner: for a
                              graph whose shape class (fastsv_tune_key) has an entry, the entry's k2_items,
                              k2_threads, col_blocks, sparse_div and batch_sparse_div replace the values above.
                              The file is read once, by fastsv_create; an unreadable file is an argument error */
} fastsv_options;

typedef struct {
    int64_t n;                 /* vertices of the last call (sum over graphs for batched calls) */
    int64_t m;                 /* directed CSR entries of the last call */
    int64_t iterations;        /* iterations executed (single-graph calls; max over graphs for batched) */
    int32_t status;            /* fastsv_status of the last call, including device-detected errors */
    int32_t converged;         /* 1 if every graph reached an unchanged f[f] */
    float ms_total;            /* device time of the last call's work on its stream (timing = 1) */
    float ms_setup;            /* of which: partitioning, state initialisation, validation */
    float ms_k2;               /* host-loop mode only: total time of the full-SpMV kernel over the
                                  timed_dense_iters iterations that ran it */
    float ms_k3;               /* host-loop mode only: total time of the grandparent kernel (timed_iters) */
    float ms_push;             /* host-loop mode only: total time of the sparse (push) iterations' SpMSpV */
    float ms_hook;             /* host-loop mode only: total time of the hooking kernel (timed_iters) */
    int32_t sparse_iters;      /* single-graph calls: iterations that pushed from the changed vertices */
    int32_t dense_iters;       /* iterations that ran the full SpMV (iterations - sparse_iters) */
    int32_t trace_len;         /* entries valid in changed_per_iter */
    int32_t col_blocks;        /* column blocks the last single-graph call used (1 = unblocked) */
    int64_t changed_per_iter[64]; /* single-graph calls: grandparents changed in iteration i */
    int32_t timed_iters;       /* host-loop mode: iterations the ms_k2 .. ms_hook fields cover.  A
                                  column-blocked call runs its first iteration before the loop, on the
                                  original CSR (no gathers are needed while gf is the identity); that
                                  iteration is part of ms_setup */
    int32_t timed_dense_iters; /* host-loop mode: of those, the iterations that ran the full SpMV */
    int32_t tuned;             /* 1 if the last call took its kernel choices from the tuning cache */
    int32_t pad0;
    int64_t block_runs;        /* column-blocked single-graph calls: runs (compressed rows) over all blocks */
} fastsv_stats;

/*
 * Shape class of a call, as the tuning cache keys it: kind 0 = single graph
 * (n vertices, m entries, rowptr_bits), kind 1 = batched call (n and m summed
 * over `graphs` graphs).  Writes a NUL-terminated string such as
 * "single n26 d10 r64" (log2 of n rounded; half-octaves of m/n) into out[cap]
 * and returns its length, or -1 for a bad argument.  The autotuner writes
 * cache lines under these keys; fastsv_cc, fastsv_cc_host and
 * fastsv_cc_batched look them up.  Pools do not: they run the handle's own
 * options.
 */
int32_t fastsv_tune_key(int32_t kind, int64_t n, int64_t m, int64_t graphs, int32_t rowptr_bits, char* out,
                        int32_t cap);

/* Fill *opt with the defaults listed above. */
void fastsv_default_options(fastsv_options* opt);

/* Create a handle on the current CUDA device.  opt may be NULL (defaults).
 * Errors: FASTSV_ERR_INVALID_ARG (out NULL, bad option), FASTSV_ERR_CUDA. */
fastsv_status fastsv_create(fastsv_t* out, const fastsv_options* opt);

/* Release the handle and its workspace (synchronises with its last stream). */
fastsv_status fastsv_destroy(fastsv_t h);

/*
 * Connected components of one graph (Algorithm 2, Section 3; result as in
 * Section 3.4).
 *   n          vertices, 0 <= n <= 2^31 - 1 (n = 0: no work, 0 iterations)
 *   row_ptr    device, n+1 entries of rowptr_bits width (int32 or int64),
 *              row_ptr[0] = 0, non-decreasing; m = row_ptr[n] directed entries
 *   col_idx    device, m int32 neighbour ids (symmetric CSR)
 *   labels_out device, n int32; receives the smallest vertex id of each
 *              vertex's component.  It also serves as the parent vector f
 *              during the solve, so it must not alias row_ptr or col_idx.
 *   stream     cudaStream_t
 * Synchronises with `stream` once, to read m = row_ptr[n] (a column-blocked
 * call once more, after its first iteration: see col_blocks).  The rest of
 * the solve is enqueued; labels_out is valid when the stream reaches the end
 * of it.
 */
fastsv_status fastsv_cc(fastsv_t h, int64_t n, const void* row_ptr, const int32_t* col_idx, int32_t* labels_out,
                        void* stream);

/*
 * fastsv_cc from host buffers: copies row_ptr and col_idx to handle-owned
 * device memory, solves, and copies the labels back, all on `stream`, and
 * returns when labels_host is filled (synchronises).  Host pointers; pinned
 * memory recommended.  Same sizes and layout as fastsv_cc.  For a
 * column-blocked graph (without validation) col_idx is copied in chunks on a
 * stream of the handle's own, and the first iteration works on every chunk
 * once it has landed; when the handle's run arrays are large enough from an
 * earlier call, every chunk is also copied into the column blocks at once
 * (the call checks the copy's totals when all chunks are in, and copies
 * again if the runs did not fit).  fastsv_get_stats' ms_total then includes
 * the copy.
 */
fastsv_status fastsv_cc_host(fastsv_t h, int64_t n, const void* row_ptr_host, const int32_t* col_idx_host,
                             int32_t* labels_host, void* stream);

/*
 * Connected components of many independent graphs in one solve: Algorithm 2
 * runs on the disjoint union, and each graph stops at its own early
 * termination (Section 3.4), so every graph gets exactly the labels and
 * iteration count it gets alone.
 *   num_graphs G >= 0
 *   vtx_off    device int64[G+1]: graph g owns batch vertices [vtx_off[g], vtx_off[g+1]), vtx_off[0] = 0
 *   edge_off   device int64[G+1]: graph g's entries are col_idx[edge_off[g] .. edge_off[g+1]), edge_off[0] = 0
 *   row_ptr    device int32[vtx_off[G] + G]: graph g's LOCAL row_ptr (n_g + 1 entries, starting at 0 and
 *              ending at m_g) at row_ptr[vtx_off[g] + g ...]
 *   col_idx    device int32[edge_off[G]]: LOCAL neighbour ids of each graph
 *   labels_out device int32[vtx_off[G]]: LOCAL labels (smallest local id of the component)
 *   iters_out  device int32[G] or NULL: iterations each graph executed
 * Synchronises once to read vtx_off[G] and edge_off[G]; the solve is enqueued.
 */
fastsv_status fastsv_cc_batched(fastsv_t h, int32_t num_graphs, const int64_t* vtx_off, const int64_t* edge_off,
                                const int32_t* row_ptr, const int32_t* col_idx, int32_t* labels_out,
                                int32_t* iters_out, void* stream);

/* Wait for the handle's last call to finish on its stream and report it.
 * Returns the call's status (FASTSV_OK, FASTSV_ERR_MAX_ITERS, ...). */
fastsv_status fastsv_get_stats(fastsv_t h, fastsv_stats* out);

/* Human-readable name of a status code (static string). */
const char* fastsv_status_string(fastsv_status s);

/* Last CUDA runtime error code seen by this handle (0 if none). */
int32_t fastsv_last_cuda_error(fastsv_t h);

/* Number of kernels this handle has launched so far, counting every kernel
 * of every iteration of the device-side loop (read after fastsv_get_stats). */
int64_t fastsv_kernel_launches(fastsv_t h);

/*
 * Serving pool (continuous batching).  A pool keeps up to max_slots graphs
 * resident in device memory within hbm_budget_bytes and advances all of them
 * together: fastsv_pool_step runs `iters` iterations of Algorithm 2 over every
 * active slot in one device-side loop, so graphs admitted between steps join
 * the running batch at an iteration boundary.  Each slot stops at its own
 * early termination (Section 3.4), so a graph's labels and iteration count do
 * not depend on what else is in the pool.
 */

/* Create the handle's pool (one per handle).  Allocates the arena and writes
 * it once (so that later host-to-device copies into it run at full speed);
 * synchronises the device. */
fastsv_status fastsv_pool_create(fastsv_t h, size_t hbm_budget_bytes, int32_t max_slots);

/* Bytes of pool memory a graph with n vertices and m directed entries uses. */
size_t fastsv_pool_bytes(int64_t n, int64_t m);

/*
 * Admit one graph: row_ptr_host int32[n+1] and col_idx_host int32[m] (host
 * memory, pinned recommended, must stay valid until the graph is harvested),
 * labels_host int32[n] host memory that receives the labels when the slot is
 * harvested.  The copies to the device are enqueued on the pool's copy
 * stream and may be issued while a step runs (they overlap it; the graph
 * joins at the next step).  *slot_out receives the slot id.
 * Errors: FASTSV_ERR_FULL if no slot or not enough budget is free now (try
 * again after harvesting), FASTSV_ERR_INVALID_ARG if it can never fit.
 */
fastsv_status fastsv_pool_add(fastsv_t h, int64_t n, const int32_t* row_ptr_host, const int32_t* col_idx_host,
                              int32_t* labels_host, int32_t* slot_out);

/* Advance every active slot by up to `iters` iterations (iters >= 1) on
 * `stream`.  Slots admitted earlier whose copies to the device have landed
 * join this step; slots whose copies are still running keep copying while it
 * runs and join a later step (so copies overlap iterations).  A step with no
 * resident graph waits for the first admitted graph's copies instead.  With
 * opt.pool_wait_copies = 1 every admitted slot joins (the step waits for all
 * their copies).  Enqueued; returns at once. */
fastsv_status fastsv_pool_step(fastsv_t h, int32_t iters, void* stream);

/*
 * Harvest: wait for the last step, copy the labels of up to `cap` slots that
 * have converged (or hit the iteration cap) into their host buffers, free
 * those slots, and return their ids in done_slots and iteration counts in
 * done_iters (may be NULL; a negative count marks a slot stopped by the
 * iteration cap).  *n_done receives the count; *n_active (may be NULL) the
 * slots still iterating.  Synchronises.
 */
fastsv_status fastsv_pool_poll(fastsv_t h, int32_t* done_slots, int32_t* done_iters, int32_t cap, int32_t* n_done,
                               int32_t* n_active);

/* Device time of the last step's phases (timing = 1): ms_out[0] waiting for
 * admission copies (only a step that had nothing else to run waits),
 * ms_out[1] admitting the joining graphs and rebuilding the tile lists,
 * ms_out[2] the iterations.  Waits for the step; all zero when timing is
 * off. */
fastsv_status fastsv_pool_step_times(fastsv_t h, float* ms_out);

/* Pool occupancy: slots in use and bytes of the budget in use. */
fastsv_status fastsv_pool_usage(fastsv_t h, int32_t* slots_used, size_t* bytes_used);

/*
 * Checkpoint and eviction (serving under memory pressure).  Between two
 * steps a slot holds Algorithm 2's state at an iteration boundary: the parent
 * vector f, the grandparents gf = f[f] and its iteration count (the snapshot
 * p equals f there, and the pool runs no sparse iterations, so nothing else
 * carries over).  fastsv_pool_evict copies that state into a host checkpoint
 * and frees the slot and its pool memory; fastsv_pool_restore admits the
 * graph again from the checkpoint, and the restored slot runs exactly the
 * iterations it would have run without the interruption: same labels, same
 * iteration count.
 */

/* Bytes of the checkpoint of a graph with n vertices (a 64-byte header, f, gf). */
size_t fastsv_pool_checkpoint_bytes(int64_t n);

/*
 * Evict `slot`: waits for the last step, copies the slot's state into
 * checkpoint_host (fastsv_pool_checkpoint_bytes(n) bytes of host memory,
 * owned by the caller, pinned recommended), takes the slot out of the device
 * loop and frees it and its pool memory.  The host buffers given when the
 * graph was added are no longer referenced.  Synchronises.
 * Errors: FASTSV_ERR_INVALID_ARG if `slot` is not a graph that has taken part
 * in a step and is still iterating (a finished graph is harvested by
 * fastsv_pool_poll; one added since the last step has no state yet).
 */
fastsv_status fastsv_pool_evict(fastsv_t h, int32_t slot, void* checkpoint_host);

/*
 * Admit a graph again from its checkpoint: arguments as fastsv_pool_add (the
 * same graph; its host buffers must stay valid until it is harvested) plus
 * the checkpoint.  The copies are enqueued on the pool's copy stream, so
 * checkpoint_host, like the graph's buffers, must stay valid until the slot
 * is harvested or evicted again.
 * Errors: as fastsv_pool_add; FASTSV_ERR_INVALID_ARG also for a checkpoint
 * whose header does not match (n, m) or is not a checkpoint.
 */
fastsv_status fastsv_pool_restore(fastsv_t h, int64_t n, const int32_t* row_ptr_host, const int32_t* col_idx_host,
                                  int32_t* labels_host, const void* checkpoint_host, int32_t* slot_out);

/*
 * Largest vertex count fastsv_cc_noalloc accepts (the size of its built-in
 * scratch: two int32 vectors of this length, 8 MiB, plus a counter, held on
 * every GPU that loads the library until the process exits).
 */
#define FASTSV_NOALLOC_MAX_VERTICES (1 << 20)

/*
 * Connected components of one graph without any device allocation by the
 * library.  (The paper has no counterpart: this is a deployment variant of
 * fastsv_cc.)  It is for callers that must not allocate device memory while
 * they run: a host framework that has reserved all device memory in its own
 * pool, where cudaMalloc would fail or fragment that pool; latency-critical
 * loops that cannot afford cudaMalloc/cudaFree, which can synchronise the
 * whole device; and code that may not call an allocator at all.  It needs no
 * handle: the per-vertex state the solve keeps lives in a fixed scratch array
 * built into the library instead of handle workspace.
 *   n          vertices, 0 <= n <= FASTSV_NOALLOC_MAX_VERTICES; a larger n
 *              returns FASTSV_ERR_UNSUPPORTED and does nothing
 *   row_ptr    device int32[n+1], row_ptr[0] = 0 (symmetric CSR as for fastsv_cc)
 *   col_idx    device int32[row_ptr[n]] (may be NULL when there are no entries)
 *   labels_out device int32[n]: the smallest vertex id of each vertex's component
 *   max_iters  iteration cap (>= 1); reaching it returns FASTSV_ERR_MAX_ITERS
 *   iterations_out  host int32 or NULL: iterations executed
 *   stream     cudaStream_t
 * Calls no cudaMalloc, cudaFree or other allocating routine.  The first call
 * on each device looks up the scratch array's device address (with that
 * device current) and caches it.  With lazy module loading (the CUDA
 * default) the library's device code, the scratch array included, is
 * loaded by that first call and takes device memory then: make the first
 * call (or load the library with CUDA_MODULE_LOADING=EAGER) before reserving
 * the device memory the caller wants to keep for itself.  The call
 * synchronises with `stream` once per iteration, so it must not be called
 * while `stream` is being captured.  All calls on a device share the one
 * scratch array, which keeps the previous call's contents (every call
 * re-initialises what it reads): calls that overlap on the GPU, from any
 * thread or stream, race on it and must be serialised by the caller.
 * The CSR is not validated: row_ptr must be non-decreasing with
 * row_ptr[0] = 0, and col_idx must hold row_ptr[n] ids; neighbour ids
 * outside [0, n) are skipped, but a malformed row_ptr makes the kernels
 * read col_idx out of bounds.  Returns when labels_out is final.
 */
fastsv_status fastsv_cc_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* labels_out,
                                int32_t max_iters, int32_t* iterations_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTSV_H */

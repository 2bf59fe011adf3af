// fastsv.cu -- libfastsv: handle, workspace, device-side iteration loop and
// the single-graph / batched entry points of include/fastsv.h.
//
// Every call runs, on the caller's stream:
//   set-up   segment table, merge-path partition of each graph into hooking
//            tiles, identity initialisation of f, p, gf (Algorithm 2, first
//            loop), optional CSR validation;
//   loop     a CUDA graph whose conditional WHILE node repeats
//            {k2_hook, k3_grandparent} until no graph's gf changed (the
//            early termination of Section 3.4) -- no host round trip per
//            iteration;
//   finish   per-graph iteration counts and a summary copied to pinned memory.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <climits>
#include <vector>

#include "fastsv_internal.h"
#include "fastsv_kernels.cuh"
#include "variants.cuh"

using namespace fsv;

namespace fsv {

fastsv_status cuda_fail(fastsv_ctx* h, cudaError_t e) {
    if (h) h->last_cuda_error = (int)e;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FASTSV_ERR_OOM : FASTSV_ERR_CUDA;
}

fastsv_status dev_alloc(fastsv_ctx* h, void** p, size_t bytes) {
    *p = nullptr;
    h->alloc_count++;
    if (h->opt.fail_alloc_after > 0 && h->alloc_count == h->opt.fail_alloc_after) return FASTSV_ERR_OOM;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(h, e);
    }
    return FASTSV_OK;
}

static void dev_free(void** p) {
    if (*p) cudaFree(*p);
    *p = nullptr;
}

static int64_t grow(int64_t need, int64_t cap) {
    int64_t c = cap + cap / 2;
    return need > c ? need : c;
}

fastsv_status ensure_workspace(fastsv_ctx* h, int64_t n, int64_t k2, int64_t k3, int64_t segs) {
    fastsv_status st;
    if (segs > h->cap_segs) {
        dev_free((void**)&h->d_segs);
        h->cap_segs = 0;
        int64_t c = grow(segs, h->cap_segs);
        if ((st = dev_alloc(h, (void**)&h->d_segs, (size_t)c * sizeof(Seg))) != FASTSV_OK) return st;
        h->cap_segs = c;
    }
    if (k2 > h->cap_k2) {
        dev_free((void**)&h->d_k2_seg);
        dev_free((void**)&h->d_k2_row);
        h->cap_k2 = 0;
        int64_t c = grow(k2 + 1, h->cap_k2);
        if ((st = dev_alloc(h, (void**)&h->d_k2_seg, (size_t)c * 4)) != FASTSV_OK) return st;
        if ((st = dev_alloc(h, (void**)&h->d_k2_row, (size_t)c * 4)) != FASTSV_OK) {
            dev_free((void**)&h->d_k2_seg);
            return st;
        }
        h->cap_k2 = c;
    }
    if (k3 > h->cap_k3) {
        dev_free((void**)&h->d_k3_seg);
        h->cap_k3 = 0;
        int64_t c = grow(k3 + 1, h->cap_k3);
        if ((st = dev_alloc(h, (void**)&h->d_k3_seg, (size_t)c * 4)) != FASTSV_OK) return st;
        h->cap_k3 = c;
    }
    if (n > h->cap_n) {
        int32_t** arrays[4] = {&h->d_p, &h->d_gf, &h->d_mngf, &h->d_frontier};
        for (auto a : arrays) dev_free((void**)a);
        h->cap_n = 0;
        int64_t c = n;
        for (auto a : arrays) {
            // the frontier holds (graph, vertex) pairs: two int32 per vertex
            const size_t bytes = (size_t)c * 4 * (a == &h->d_frontier ? 2 : 1);
            if ((st = dev_alloc(h, (void**)a, bytes)) != FASTSV_OK) {
                for (auto b : arrays) dev_free((void**)b);
                return st;
            }
        }
        h->cap_n = c;
    }
    return FASTSV_OK;
}

// merge-path tile shape of the SpMV (threads x items per thread): 64 or
// 256 threads, 4, 8 or 16 items
int k2_items(const fastsv_ctx* h) {
    int it = h->opt.k2_items;
    return (it == 4 || it == 8 || it == 16) ? it : 8;
}

int k2_threads(const fastsv_ctx* h) {
    int t = h->opt.k2_threads;
    return (t == 64 || t == 256) ? t : 256;
}

int64_t k2_tile(const fastsv_ctx* h) { return (int64_t)k2_threads(h) * k2_items(h); }

// kernel instance selection -------------------------------------------------

template <typename RP, int THREADS>
static const void* k2_func_t(int items) {
    if (items == 4) return (const void*)k2_spmv<RP, THREADS, 4>;
    if (items == 16) return (const void*)k2_spmv<RP, THREADS, 16>;
    return (const void*)k2_spmv<RP, THREADS, 8>;
}

static const void* k2_func(int rp64, int items, int threads) {
    if (rp64) return threads == 256 ? k2_func_t<int64_t, 256>(items) : k2_func_t<int64_t, 64>(items);
    return threads == 256 ? k2_func_t<int32_t, 256>(items) : k2_func_t<int32_t, 64>(items);
}

static int k2_smem(int items, int threads) {
    if (threads == 256)
        return items == 4 ? k2_smem_bytes<256, 4>() : items == 16 ? k2_smem_bytes<256, 16>() : k2_smem_bytes<256, 8>();
    return items == 4 ? k2_smem_bytes<64, 4>() : items == 16 ? k2_smem_bytes<64, 16>() : k2_smem_bytes<64, 8>();
}

static fastsv_status k2_grid_for(fastsv_ctx* h, int rp64, int items, int threads, int* grid) {
    const void* fn = k2_func(rp64, items, threads);
    int smem = k2_smem(items, threads);
    FSV_CUDA(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    FSV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    if (per_sm < 1) per_sm = 1;
    if (h->opt.grid_ctas_per_sm > 0 && h->opt.grid_ctas_per_sm < per_sm) per_sm = h->opt.grid_ctas_per_sm;
    *grid = per_sm * h->num_sms;
    return FASTSV_OK;
}


// kernel functions of one iteration for a given configuration
struct IterKernels {
    const void* spmv;
    const void* push;
    const void* hook;
    const void* k3;
    int spmv_smem;
    int spmv_grid, vtx_grid;
};

static fastsv_status iter_kernels(fastsv_ctx* h, int rp64_orig, int rp64_dense, int items, IterKernels* k) {
    const int threads = k2_threads(h);
    k->spmv = k2_func(rp64_dense, items, threads);
    k->spmv_smem = k2_smem(items, threads);
    k->push = rp64_orig ? (const void*)k2_push<int64_t> : (const void*)k2_push<int32_t>;
    k->hook = (const void*)k2_hook;
    k->k3 = rp64_orig ? (const void*)k3_grandparent<int64_t> : (const void*)k3_grandparent<int32_t>;
    fastsv_status st;
    if ((st = k2_grid_for(h, rp64_dense, items, threads, &k->spmv_grid)) != FASTSV_OK) return st;
    int per_sm = 0;
    FSV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k->k3, K3_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    if (h->opt.grid_ctas_per_sm > 0 && h->opt.grid_ctas_per_sm < per_sm) per_sm = h->opt.grid_ctas_per_sm;
    k->vtx_grid = per_sm * h->num_sms;
    return FASTSV_OK;
}

// the device-side loop:
//   WHILE(cond) { k_iter_begin; k2_spmv | k2_push; k2_hook; k3_grandparent }
// (k2_spmv and k2_push read the iteration's mode and return at once when it
// is not theirs)
fastsv_status get_loop_graph(fastsv_ctx* h, Ctx* ctx, int rp64_orig, int rp64_dense, int items, int nblocks,
                             LoopGraph** out) {
    const int threads = k2_threads(h);
    GraphKey key{rp64_orig * 2 + rp64_dense, items * 1000 + threads, h->opt.mode * 64 + nblocks, ctx};
    auto it = h->graphs.find(key);
    if (it != h->graphs.end()) {
        *out = &it->second;
        return FASTSV_OK;
    }
    IterKernels K;
    fastsv_status st = iter_kernels(h, rp64_orig, rp64_dense, items, &K);
    if (st != FASTSV_OK) return st;
    LoopGraph lg;
    FSV_CUDA(h, cudaGraphCreate(&lg.graph, 0));
    FSV_CUDA(h, cudaGraphConditionalHandleCreate(&lg.cond, lg.graph, 1, cudaGraphCondAssignDefault));
    // the struct holds a union of node kinds and has no usable default
    // constructor: start from zeroed storage
    alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
    memset(cp_storage, 0, sizeof(cp_storage));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = lg.cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond_node;
    FSV_CUDA(h, cudaGraphAddNode(&cond_node, lg.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    cudaGraphConditionalHandle cond = lg.cond;
    int use_cond = 1;
    void* a_begin[] = {(void*)&ctx, (void*)&cond, (void*)&use_cond};
    void* a_ctx[] = {(void*)&ctx};
    void* a_k3[] = {(void*)&ctx, (void*)&cond, (void*)&use_cond};
    // one SpMV node for an unblocked solve (block = -1), else one per column
    // block, in order (kernel parameters are copied when a node is added)
    std::vector<int> blocks;
    if (nblocks <= 0)
        blocks.push_back(-1);
    else
        for (int b = 0; b < nblocks; ++b) blocks.push_back(b);
    std::vector<void*> spmv_args(2 * blocks.size());
    struct NodeSpec {
        const void* fn;
        int grid, block, smem;
        void** args;
    };
    std::vector<NodeSpec> nodes;
    nodes.push_back({(const void*)k_iter_begin, K.vtx_grid, 256, 0, a_begin});
    for (size_t i = 0; i < blocks.size(); ++i) {
        spmv_args[2 * i] = (void*)&ctx;
        spmv_args[2 * i + 1] = (void*)&blocks[i];
        nodes.push_back({K.spmv, K.spmv_grid, threads, K.spmv_smem, &spmv_args[2 * i]});
    }
    nodes.push_back({K.push, h->num_sms * 8, 256, 0, a_ctx});
    nodes.push_back({K.hook, K.vtx_grid, K3_THREADS, 0, a_ctx});
    nodes.push_back({K.k3, K.vtx_grid, K3_THREADS, 0, a_k3});
    cudaGraphNode_t prev = nullptr;
    for (size_t i = 0; i < nodes.size(); ++i) {
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        kp.func = (void*)nodes[i].fn;
        kp.gridDim = dim3((unsigned)nodes[i].grid);
        kp.blockDim = dim3((unsigned)nodes[i].block);
        kp.sharedMemBytes = (unsigned)nodes[i].smem;
        kp.kernelParams = nodes[i].args;
        cudaGraphNode_t node;
        FSV_CUDA(h, cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
        prev = node;
    }
    FSV_CUDA(h, cudaGraphInstantiate(&lg.exec, lg.graph, 0));
    auto res = h->graphs.emplace(key, lg);
    *out = &res.first->second;
    return FASTSV_OK;
}

fastsv_status run_loop(fastsv_ctx* h, Ctx* ctx, int rp64_orig, int rp64_dense, int items, int nblocks,
                       cudaStream_t s) {
    const int spmv_launches = nblocks > 0 ? nblocks : 1;
    if (h->opt.use_graph) {
        LoopGraph* lg = nullptr;
        fastsv_status st = get_loop_graph(h, ctx, rp64_orig, rp64_dense, items, nblocks, &lg);
        if (st != FASTSV_OK) return st;
        FSV_CUDA(h, cudaGraphLaunch(lg->exec, s));
        h->pending_loop_kernels = 4 + spmv_launches;
        return FASTSV_OK;
    }
    // host loop: one synchronisation per iteration, per-kernel event timing
    IterKernels K;
    fastsv_status st = iter_kernels(h, rp64_orig, rp64_dense, items, &K);
    if (st != FASTSV_OK) return st;
    const int threads = k2_threads(h);
    cudaEvent_t e[5];
    for (int i = 0; i < 5; ++i) FSV_CUDA(h, cudaEventCreate(&e[i]));
    float t_spmv = 0.f, t_push = 0.f, t_hook = 0.f, t_k3 = 0.f;
    int iters = 0, dense = 0;
    cudaGraphConditionalHandle none = 0;
    int no_cond = 0;
    int32_t limit = h->loop_limit_host;
    fastsv_status rc = FASTSV_OK;
    int32_t mode = MODE_DENSE;
    for (;;) {
        void* a_begin[] = {(void*)&ctx, (void*)&none, (void*)&no_cond};
        void* a_ctx[] = {(void*)&ctx};
        void* a_k3[] = {(void*)&ctx, (void*)&none, (void*)&no_cond};
        cudaError_t ce = cudaEventRecord(e[0], s);
        if (ce == cudaSuccess)
            ce = cudaLaunchKernel((const void*)k_iter_begin, dim3(K.vtx_grid), dim3(256), a_begin, 0, s);
        for (int b = 0; b < spmv_launches && ce == cudaSuccess; ++b) {
            int blk = nblocks > 0 ? b : -1;
            void* a_spmv[] = {(void*)&ctx, (void*)&blk};
            ce = cudaLaunchKernel(K.spmv, dim3(K.spmv_grid), dim3(threads), a_spmv, K.spmv_smem, s);
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(e[1], s);
        if (ce == cudaSuccess) ce = cudaLaunchKernel(K.push, dim3(h->num_sms * 8), dim3(256), a_ctx, 0, s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e[2], s);
        if (ce == cudaSuccess) ce = cudaLaunchKernel(K.hook, dim3(K.vtx_grid), dim3(K3_THREADS), a_ctx, 0, s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e[3], s);
        if (ce == cudaSuccess) ce = cudaLaunchKernel(K.k3, dim3(K.vtx_grid), dim3(K3_THREADS), a_k3, 0, s);
        if (ce == cudaSuccess) ce = cudaEventRecord(e[4], s);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(h->h_scalar, &ctx->any_active, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync((int32_t*)h->h_scalar + 1, &ctx->mode, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
            rc = cuda_fail(h, ce);
            break;
        }
        h->launches += 4 + spmv_launches;
        float a = 0.f, b = 0.f, c = 0.f, d = 0.f;
        cudaEventElapsedTime(&a, e[0], e[1]);
        cudaEventElapsedTime(&b, e[1], e[2]);
        cudaEventElapsedTime(&c, e[2], e[3]);
        cudaEventElapsedTime(&d, e[3], e[4]);
        if (mode & MODE_DENSE) {
            t_spmv += a;
            ++dense;
        }
        if (mode & MODE_PUSH) t_push += b;
        t_hook += c;
        t_k3 += d;
        ++iters;
        mode = ((int32_t*)h->h_scalar)[1];  // the mode k3 chose for the next iteration
        if (((int32_t*)h->h_scalar)[0] == 0 || iters >= limit) break;
    }
    for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
    h->ms_k2 = t_spmv;
    h->ms_push = t_push;
    h->ms_hook = t_hook;
    h->ms_k3 = t_k3;
    h->dense_iters = dense;
    h->timed_iters = iters;
    h->pending_loop_kernels = 0;
    return rc;
}

// ---------------------------------------------------------------------------
// convergence ablation sv1..sv4: host loop, one synchronisation per iteration
// ---------------------------------------------------------------------------

static fastsv_status run_variant_loop(fastsv_ctx* h, Ctx* ctx, int rp64, int items, int variant, int64_t n,
                                      int32_t* f, cudaStream_t s) {
    IterKernels K;
    fastsv_status st = iter_kernels(h, rp64, rp64, items, &K);
    if (st != FASTSV_OK) return st;
    const int threads = k2_threads(h);
    const int vgrid = h->num_sms * 8;
    VarPtrs P{f, h->d_p, h->d_gf, h->d_mngf, &h->d_segs[0].changed, n};
    const int root_test = variant <= 2, aggressive = variant == 4, two_phase = variant <= 3;
    cudaEvent_t e[3];
    for (int i = 0; i < 3; ++i) FSV_CUDA(h, cudaEventCreate(&e[i]));
    float t_spmv = 0.f, t_rest = 0.f;
    int iters = 0;
    cudaGraphConditionalHandle none = 0;
    int no_cond = 0, blk = -1;
    fastsv_status rc = FASTSV_OK;
    for (;;) {
        void* a_begin[] = {(void*)&ctx, (void*)&none, (void*)&no_cond};
        void* a_spmv[] = {(void*)&ctx, (void*)&blk};
        void* a_hook[] = {(void*)&P, (void*)&root_test, (void*)&aggressive};
        void* a_p[] = {(void*)&P};
        void* a_commit[] = {(void*)&P, (void*)&two_phase};
        void* a_close[] = {(void*)&ctx, (void*)&none, (void*)&no_cond};
        int launched = 0;
        cudaError_t ce = cudaEventRecord(e[0], s);
        if (ce == cudaSuccess)
            ce = cudaLaunchKernel((const void*)k_iter_begin, dim3(K.vtx_grid), dim3(256), a_begin, 0, s), ++launched;
        if (ce == cudaSuccess)
            ce = cudaLaunchKernel(K.spmv, dim3(K.spmv_grid), dim3(threads), a_spmv, K.spmv_smem, s), ++launched;
        if (ce == cudaSuccess) ce = cudaEventRecord(e[1], s);
        if (ce == cudaSuccess)
            ce = cudaLaunchKernel((const void*)kv_hook, dim3(vgrid), dim3(256), a_hook, 0, s), ++launched;
        if (ce == cudaSuccess && two_phase)
            ce = cudaLaunchKernel((const void*)kv_shortcut, dim3(vgrid), dim3(256), a_p, 0, s), ++launched;
        if (ce == cudaSuccess)
            ce = cudaLaunchKernel((const void*)kv_commit, dim3(vgrid), dim3(256), a_commit, 0, s), ++launched;
        if (ce == cudaSuccess)
            ce = cudaLaunchKernel((const void*)kv_grand, dim3(vgrid), dim3(256), a_p, 0, s), ++launched;
        if (ce == cudaSuccess)
            ce = cudaLaunchKernel((const void*)k_close, dim3(1), dim3(256), a_close, 0, s), ++launched;
        if (ce == cudaSuccess) ce = cudaEventRecord(e[2], s);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(h->h_scalar, &ctx->any_active, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        h->launches += launched;
        if (ce != cudaSuccess) {
            rc = cuda_fail(h, ce);
            break;
        }
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, e[0], e[1]);
        cudaEventElapsedTime(&b, e[1], e[2]);
        t_spmv += a;
        t_rest += b;
        ++iters;
        if (((int32_t*)h->h_scalar)[0] == 0 || iters >= h->loop_limit_host) break;
    }
    for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]);
    h->ms_k2 = t_spmv;
    h->ms_hook = t_rest;
    h->dense_iters = iters;
    h->timed_iters = iters;
    h->pending_loop_kernels = 0;
    return rc;
}

// ---------------------------------------------------------------------------
// asynchronous mode: {k_async, k_close} per iteration, in a device WHILE loop
// (or a host loop when use_graph = 0)
// ---------------------------------------------------------------------------

constexpr int ASYNC_THREADS = 256, ASYNC_ITEMS = 8;

static const void* async_func(int rp64) {
    return rp64 ? (const void*)k_async<int64_t, ASYNC_THREADS, ASYNC_ITEMS>
                : (const void*)k_async<int32_t, ASYNC_THREADS, ASYNC_ITEMS>;
}

static fastsv_status run_async_loop(fastsv_ctx* h, Ctx* ctx, int rp64, cudaStream_t s) {
    const void* fn = async_func(rp64);
    const int smem = async_smem_bytes<ASYNC_THREADS, ASYNC_ITEMS>();
    FSV_CUDA(h, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    FSV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ASYNC_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    if (h->opt.grid_ctas_per_sm > 0 && h->opt.grid_ctas_per_sm < per_sm) per_sm = h->opt.grid_ctas_per_sm;
    const int grid = per_sm * h->num_sms;
    if (h->opt.use_graph) {
        GraphKey key{rp64 * 2 + rp64, ASYNC_ITEMS * 1000 + ASYNC_THREADS, FASTSV_MODE_ASYNC * 64, ctx};
        auto it = h->graphs.find(key);
        if (it == h->graphs.end()) {
            LoopGraph lg;
            FSV_CUDA(h, cudaGraphCreate(&lg.graph, 0));
            FSV_CUDA(h, cudaGraphConditionalHandleCreate(&lg.cond, lg.graph, 1, cudaGraphCondAssignDefault));
            alignas(cudaGraphNodeParams) unsigned char cp_storage[sizeof(cudaGraphNodeParams)];
            memset(cp_storage, 0, sizeof(cp_storage));
            cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_storage);
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = lg.cond;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cond_node;
            FSV_CUDA(h, cudaGraphAddNode(&cond_node, lg.graph, nullptr, nullptr, 0, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            cudaGraphConditionalHandle cond = lg.cond;
            int use_cond = 1;
            void* a_async[] = {(void*)&ctx};
            void* a_close[] = {(void*)&ctx, (void*)&cond, (void*)&use_cond};
            cudaKernelNodeParams kp;
            memset(&kp, 0, sizeof(kp));
            kp.func = (void*)fn;
            kp.gridDim = dim3((unsigned)grid);
            kp.blockDim = dim3(ASYNC_THREADS);
            kp.sharedMemBytes = (unsigned)smem;
            kp.kernelParams = a_async;
            cudaGraphNode_t n1, n2;
            FSV_CUDA(h, cudaGraphAddKernelNode(&n1, body, nullptr, 0, &kp));
            memset(&kp, 0, sizeof(kp));
            kp.func = (void*)k_close;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(256);
            kp.kernelParams = a_close;
            FSV_CUDA(h, cudaGraphAddKernelNode(&n2, body, &n1, 1, &kp));
            FSV_CUDA(h, cudaGraphInstantiate(&lg.exec, lg.graph, 0));
            it = h->graphs.emplace(key, lg).first;
        }
        FSV_CUDA(h, cudaGraphLaunch(it->second.exec, s));
        h->pending_loop_kernels = 2;
        return FASTSV_OK;
    }
    cudaGraphConditionalHandle none = 0;
    int no_cond = 0, iters = 0;
    for (;;) {
        void* a_async[] = {(void*)&ctx};
        void* a_close[] = {(void*)&ctx, (void*)&none, (void*)&no_cond};
        cudaError_t ce = cudaLaunchKernel(fn, dim3(grid), dim3(ASYNC_THREADS), a_async, smem, s);
        if (ce == cudaSuccess) ce = cudaLaunchKernel((const void*)k_close, dim3(1), dim3(256), a_close, 0, s);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(h->h_scalar, &ctx->any_active, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_fail(h, ce);
        h->launches += 2;
        ++iters;
        if (((int32_t*)h->h_scalar)[0] == 0 || iters >= h->loop_limit_host) break;
    }
    h->pending_loop_kernels = 0;
    return FASTSV_OK;
}

int setup_grid(const fastsv_ctx* h) { return h->num_sms * 8; }

// prefix sums of tile counts, merge-path partition, identity state of
// segments that have not iterated yet (int32 row pointers)
fastsv_status rebuild_tiles(fastsv_ctx* h, Ctx* ctx, cudaStream_t s) {
    k_scan_tiles<<<1, 1024, 0, s>>>(ctx);
    k_partition<int32_t><<<setup_grid(h), 256, 0, s>>>(ctx);
    k_init_state<<<setup_grid(h), 256, 0, s>>>(ctx);
    h->launches += 3;
    FSV_CUDA(h, cudaGetLastError());
    return FASTSV_OK;
}

// stream ordering between consecutive calls of one handle
static void order_after_previous(fastsv_ctx* h, cudaStream_t s) {
    if (h->pending && h->last_stream != s) cudaStreamWaitEvent(s, h->ev_end, 0);
}

static fastsv_status finish_call(fastsv_ctx* h, cudaStream_t s, int32_t* iters_out, int64_t n, int64_t m,
                                 bool single) {
    k_finish<<<1, 256, 0, s>>>(h->d_ctx, iters_out, h->pending_loop_kernels);
    // launches made from the host count now; the device loop's count arrives
    // with the summary
    h->launches += h->pending_fixed_launches + 1;
    h->pending_fixed_launches = 0;
    FSV_CUDA(h, cudaGetLastError());
    FSV_CUDA(h, cudaMemcpyAsync(h->h_sum, &h->d_ctx->sum, sizeof(Summary), cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaEventRecord(h->ev_end, s));
    h->pending = true;
    h->last_stream = s;
    h->last_n = n;
    h->last_m = m;
    h->single = single;
    return FASTSV_OK;
}

// validation needs its result before any hooking kernel reads the graph
static fastsv_status run_validation(fastsv_ctx* h, int rp64, cudaStream_t s) {
    if (!h->opt.validate) return FASTSV_OK;
    if (rp64)
        k_validate<int64_t><<<setup_grid(h), 256, 0, s>>>(h->d_ctx, h->opt.validate >= 2);
    else
        k_validate<int32_t><<<setup_grid(h), 256, 0, s>>>(h->d_ctx, h->opt.validate >= 2);
    h->pending_fixed_launches += 1;
    FSV_CUDA(h, cudaGetLastError());
    FSV_CUDA(h, cudaMemcpyAsync(h->h_scalar, &h->d_ctx->val_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaStreamSynchronize(s));
    if (*(int32_t*)h->h_scalar != 0) {
        h->launches += h->pending_fixed_launches;
        h->pending_fixed_launches = 0;
        h->last_status = FASTSV_ERR_INVALID_GRAPH;
        h->pending = false;
        return FASTSV_ERR_INVALID_GRAPH;
    }
    return FASTSV_OK;
}

// number of column blocks for a graph (1 = unblocked): the grandparent
// vector must be larger than the L2 share given to one block's slice, and the
// graph dense enough that the per-block runs and the one-time copy pay off
static int choose_col_blocks(const fastsv_ctx* h, int64_t n, int64_t m) {
    int nb = h->opt.col_blocks;
    if (m > (int64_t)INT32_MAX - 1) return 1;  // block entry offsets are int32
    if (nb == 1) return 1;
    if (nb <= 0) {
        // Automatic: block when the gathered vector (4n bytes) is at least
        // 1.5x the L2 and the graph is dense enough (m >= 8n), one block per
        // col_block_mib MiB of the gathered vector (default 64: measured on
        // GB300 at R-MAT scale 26, 4 blocks solve in 51.4 ms, 8 in 52.5, 16 in
        // 59.4 (the copy's run lists grow with the block count), unblocked
        // in 70.0).
        const int64_t l2 = h->l2_bytes > 0 ? h->l2_bytes : (int64_t)129 << 20;
        if (m < 8 * n || 2 * (4 * n) < 3 * l2) return 1;
        const int64_t mib = h->opt.col_block_mib > 0 ? h->opt.col_block_mib : 64;
        const int64_t slice = mib << 20;
        const int64_t want = (4 * n + slice - 1) / slice;
        return (int)(want < 2 ? 2 : (want < MAX_COL_BLOCKS ? want : MAX_COL_BLOCKS));
    }
    if (nb > MAX_COL_BLOCKS) nb = MAX_COL_BLOCKS;
    return nb;
}

// counts (2 nb rows of tiles + 1), scan sums, the block copy's entries, the
// chunks' layouts and totals, and the host-visible checks; the runs' arrays
// grow once their count is known
static fastsv_status ensure_block_workspace(fastsv_ctx* h, int nb, int64_t tiles, int64_t m) {
    fastsv_status st;
    if (!h->d_build_scalars) {
        if ((st = dev_alloc(h, (void**)&h->d_build_scalars, 8 * 4)) != FASTSV_OK) return st;
    }
    if (!h->d_clay) {
        if ((st = dev_alloc(h, (void**)&h->d_clay, sizeof(ChunkLayout) * MAX_FEED_CHUNKS)) != FASTSV_OK) return st;
    }
    if (!h->d_ctot) {
        if ((st = dev_alloc(h, (void**)&h->d_ctot, 4 * 2 * MAX_COL_BLOCKS * MAX_FEED_CHUNKS)) != FASTSV_OK) return st;
    }
    const int64_t T1 = tiles + 1;
    const int64_t cells = 2 * (int64_t)nb * T1;
    if (cells > h->cap_blk) {
        dev_free((void**)&h->d_counts);
        h->cap_blk = 0;
        if ((st = dev_alloc(h, (void**)&h->d_counts, (size_t)cells * 4)) != FASTSV_OK) return st;
        h->cap_blk = cells;
    }
    const int64_t sums = 2 * (int64_t)nb * ((T1 + SCAN_CHUNK - 1) / SCAN_CHUNK) + 1;
    if (sums > h->cap_sums) {
        dev_free((void**)&h->d_sums);
        h->cap_sums = 0;
        if ((st = dev_alloc(h, (void**)&h->d_sums, (size_t)sums * 4)) != FASTSV_OK) return st;
        h->cap_sums = sums;
    }
    if (m > h->cap_colB) {
        dev_free((void**)&h->d_colB);
        h->cap_colB = 0;
        if ((st = dev_alloc(h, (void**)&h->d_colB, (size_t)m * 4)) != FASTSV_OK) return st;
        h->cap_colB = m;
    }
    return FASTSV_OK;
}

// rowsB / endsB for `runs` runs and `slots` leading slots (one per (chunk,
// block) pair)
static fastsv_status ensure_run_workspace(fastsv_ctx* h, int64_t runs, int64_t slots) {
    fastsv_status st;
    if (runs + slots > h->cap_runs) {
        dev_free((void**)&h->d_rowsB);
        dev_free((void**)&h->d_endsB);
        h->cap_runs = 0;
        const int64_t c = runs + runs / 8 + slots;  // room to grow a little between calls
        if ((st = dev_alloc(h, (void**)&h->d_rowsB, (size_t)c * 4)) != FASTSV_OK) return st;
        if ((st = dev_alloc(h, (void**)&h->d_endsB, (size_t)c * 4)) != FASTSV_OK) {
            dev_free((void**)&h->d_rowsB);
            return st;
        }
        h->cap_runs = c;
    }
    return FASTSV_OK;
}

// col_idx of a fastsv_cc_host call still in host memory: the first iteration
// of a column-blocked solve reads it chunk by chunk as the copies land
struct HostFeed {
    const int32_t* ci_host;  // source
    int32_t* ci_dev;         // destination (the handle's device copy)
};
constexpr int FEED_CHUNKS = 8;

static fastsv_status ensure_feed(fastsv_ctx* h) {
    if (!h->feed_stream) FSV_CUDA(h, cudaStreamCreateWithFlags(&h->feed_stream, cudaStreamNonBlocking));
    for (int i = 0; i <= FEED_CHUNKS; ++i)
        if (!h->feed_ev[i]) FSV_CUDA(h, cudaEventCreateWithFlags(&h->feed_ev[i], cudaEventDisableTiming));
    if (!h->d_feed_tiles) {
        fastsv_status st = dev_alloc(h, (void**)&h->d_feed_tiles, sizeof(int64_t) * (MAX_FEED_CHUNKS + 1));
        if (st != FASTSV_OK) return st;
    }
    return FASTSV_OK;
}

// The column-block copy of one chunk of the first iteration's tiles (range:
// the chunks' tile bounds on the device, or null for one chunk of every
// tile): scan the chunk's counts, place its blocks, and (when the runs'
// arrays are already there) split its entries into them.
struct BlockBuild {
    int nb, shift, chunks;
    int64_t tiles, m;
    const int64_t* range;
};

template <typename RP>
static fastsv_status launch_chunk_split(fastsv_ctx* h, const BlockBuild& B, int c, cudaStream_t s) {
    int per_sm = 0;
    FSV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)k_block_split<RP>, SPLIT_THREADS, 0));
    const int grid = (per_sm > 0 ? per_sm : 1) * h->num_sms;
    k_block_split<RP><<<grid, SPLIT_THREADS, 0, s>>>(h->d_ctx, h->d_clay, c, B.nb, B.shift, B.tiles + 1, B.range,
                                                    h->d_counts, h->d_colB, h->d_rowsB, h->d_endsB, B.m, h->cap_runs);
    h->pending_fixed_launches += 1;
    FSV_CUDA(h, cudaGetLastError());
    return FASTSV_OK;
}

static fastsv_status launch_chunk_layout(fastsv_ctx* h, const BlockBuild& B, int c, cudaStream_t s) {
    const int64_t T1 = B.tiles + 1;
    const int rows = 2 * B.nb;
    const int pieces = (int)((T1 + SCAN_CHUNK - 1) / SCAN_CHUNK);
    int32_t* tot = h->d_ctot + (int64_t)c * rows;
    k_scan_chunk_sums<<<(unsigned)(rows * pieces), SCAN_THREADS, 0, s>>>(h->d_counts, T1, pieces, h->d_sums, B.range, c);
    k_scan_sums<<<rows, 1024, 0, s>>>(h->d_sums, pieces, tot);
    k_scan_apply<<<(unsigned)(rows * pieces), SCAN_THREADS, 0, s>>>(h->d_counts, h->d_counts, T1, pieces, h->d_sums,
                                                                  B.range, c);
    k_chunk_layout<<<1, 32, 0, s>>>(h->d_ctx, tot, B.nb, B.range, c, h->d_clay);
    h->pending_fixed_launches += 4;
    FSV_CUDA(h, cudaGetLastError());
    return FASTSV_OK;
}

// The first iteration's hooks and grandparents, once its SpMV (every chunk
// of it) is enqueued on s, on a stream of their own: they touch none of what
// the block copy reads or writes, so they run beside it (build_blocks joins
// them before the blocks become segments).
static fastsv_status launch_first_hooks(fastsv_ctx* h, const IterKernels& K, cudaStream_t s) {
    if (!h->side_stream) FSV_CUDA(h, cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& ev : h->side_ev)
        if (!ev) FSV_CUDA(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    Ctx* ctx = h->d_ctx;
    cudaGraphConditionalHandle none = 0;
    int no_cond = 0;
    void* a_ctx[] = {(void*)&ctx};
    void* a_k3[] = {(void*)&ctx, (void*)&none, (void*)&no_cond};
    FSV_CUDA(h, cudaEventRecord(h->side_ev[0], s));
    FSV_CUDA(h, cudaStreamWaitEvent(h->side_stream, h->side_ev[0], 0));
    FSV_CUDA(h, cudaLaunchKernel(K.hook, dim3(K.vtx_grid), dim3(K3_THREADS), a_ctx, 0, h->side_stream));
    FSV_CUDA(h, cudaLaunchKernel(K.k3, dim3(K.vtx_grid), dim3(K3_THREADS), a_k3, 0, h->side_stream));
    FSV_CUDA(h, cudaEventRecord(h->side_ev[1], h->side_stream));
    h->pending_fixed_launches += 2;
    return FASTSV_OK;
}

// one iteration on segment 0's own tiles (BUILD_TILE items each), launched
// kernel by kernel: the first iteration of a column-blocked solve.  Its SpMV
// (k2_first) gathers nothing, so the per-tile merge-path search is most of
// its work: 64 threads x 16 items spend one search on 16 items.  It also
// counts every tile's entries and runs per column block for the block copy.
// Fed from host memory (feed), col_idx arrives in FEED_CHUNKS pieces and
// every piece's tiles run once it has landed; with `pipelined`, every
// chunk's block copy follows right behind (its runs' arrays are sized from
// an earlier call of the handle and checked afterwards).
template <typename RP>
static fastsv_status first_iteration_unblocked(fastsv_ctx* h, const BlockBuild& B, const HostFeed* feed,
                                               bool pipelined, cudaStream_t s) {
    const int rp64 = sizeof(RP) == 8;
    IterKernels K;
    fastsv_status st = iter_kernels(h, rp64, rp64, 8, &K);
    if (st != FASTSV_OK) return st;
    const void* spmv = (const void*)k2_first<RP>;
    const int smem = k2_first_smem();
    int per_sm = 0;
    FSV_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmv, FIRST_THREADS, smem));
    const int grid = (per_sm > 0 ? per_sm : 1) * h->num_sms;
    Ctx* ctx = h->d_ctx;
    int32_t* cnt = h->d_counts;
    int nb = B.nb, shift = B.shift;
    cudaGraphConditionalHandle none = 0;
    int no_cond = 0;
    void* a_begin[] = {(void*)&ctx, (void*)&none, (void*)&no_cond};
    FSV_CUDA(h, cudaLaunchKernel((const void*)k_iter_begin, dim3(K.vtx_grid), dim3(256), a_begin, 0, s));
    h->pending_fixed_launches += 1;
    if (!feed) {
        const int64_t* range = nullptr;
        int chunk = 0;
        void* a_spmv[] = {(void*)&ctx, (void*)&cnt, (void*)&nb, (void*)&shift, (void*)&range, (void*)&chunk};
        FSV_CUDA(h, cudaLaunchKernel(spmv, dim3(grid), dim3(FIRST_THREADS), a_spmv, smem, s));
        h->pending_fixed_launches += 1;
        if ((st = launch_first_hooks(h, K, s)) != FASTSV_OK) return st;
    } else {
        // col_idx arrives in FEED_CHUNKS copies on the feed stream (after
        // everything enqueued on s so far); every chunk's tiles run as soon as
        // their entries have landed
        if ((st = ensure_feed(h)) != FASTSV_OK) return st;
        FeedBounds fb;
        memset(&fb, 0, sizeof(fb));
        fb.chunks = FEED_CHUNKS;
        for (int c = 0; c <= FEED_CHUNKS; ++c) fb.b[c] = B.m * c / FEED_CHUNKS;
        k_feed_tiles<<<1, 32, 0, s>>>(ctx, fb, h->d_feed_tiles);
        FSV_CUDA(h, cudaEventRecord(h->feed_ev[0], s));
        FSV_CUDA(h, cudaStreamWaitEvent(h->feed_stream, h->feed_ev[0], 0));
        for (int c = 0; c < FEED_CHUNKS; ++c) {
            const int64_t e0 = fb.b[c], e1 = fb.b[c + 1];
            if (e1 > e0)
                FSV_CUDA(h, cudaMemcpyAsync(feed->ci_dev + e0, feed->ci_host + e0, (size_t)(e1 - e0) * 4,
                                            cudaMemcpyHostToDevice, h->feed_stream));
            FSV_CUDA(h, cudaEventRecord(h->feed_ev[1 + c], h->feed_stream));
        }
        const int64_t* range = h->d_feed_tiles;
        for (int c = 0; c < FEED_CHUNKS; ++c) {
            FSV_CUDA(h, cudaStreamWaitEvent(s, h->feed_ev[1 + c], 0));
            int chunk = c;
            void* a_spmv[] = {(void*)&ctx, (void*)&cnt, (void*)&nb, (void*)&shift, (void*)&range, (void*)&chunk};
            FSV_CUDA(h, cudaLaunchKernel(spmv, dim3(grid), dim3(FIRST_THREADS), a_spmv, smem, s));
            if (c == FEED_CHUNKS - 1 && (st = launch_first_hooks(h, K, s)) != FASTSV_OK) return st;
            if (pipelined) {
                if ((st = launch_chunk_layout(h, B, c, s)) != FASTSV_OK) return st;
                if ((st = launch_chunk_split<RP>(h, B, c, s)) != FASTSV_OK) return st;
            }
        }
        h->pending_fixed_launches += 1 + FEED_CHUNKS;
    }
    return FASTSV_OK;
}

// The block copy after the first iteration counted it.  Unless the chunks
// were already copied (pipelined): scan the counts over all tiles (one
// chunk), place the blocks, and split the entries.  Either way the host
// reads the copy's totals (one synchronisation: the runs' arrays are sized,
// or checked, by them), and the blocks become segments 1 .. nb C with their
// own merge-path tiles.
template <typename RP>
static fastsv_status build_blocks(fastsv_ctx* h, const BlockBuild& B, bool pipelined, int32_t tile, cudaStream_t s) {
    fastsv_status st;
    const int C = pipelined ? B.chunks : 1;
    BlockBuild one = B;
    if (!pipelined) {
        one.chunks = 1;
        one.range = nullptr;
        if ((st = launch_chunk_layout(h, one, 0, s)) != FASTSV_OK) return st;
    }
    k_chunk_check<<<1, 32, 0, s>>>(h->d_clay, C, B.nb, h->d_build_scalars);
    h->pending_fixed_launches += 1;
    FSV_CUDA(h, cudaGetLastError());
    FSV_CUDA(h, cudaMemcpyAsync(h->h_scalar, h->d_build_scalars, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaStreamSynchronize(s));
    // an error return leaves s (and so every later call) after the first
    // iteration's hooks on the side stream
    auto fail = [&](fastsv_status e) {
        cudaStreamWaitEvent(s, h->side_ev[1], 0);
        return e;
    };
    const int64_t ends = h->h_scalar[0], runs = h->h_scalar[1], contiguous = h->h_scalar[2];
    if (ends != B.m || !contiguous) return fail(FASTSV_ERR_INVALID_GRAPH);  // row_ptr not a valid CSR of m entries
    const int64_t slots = (int64_t)B.nb * C;
    const bool fits = pipelined && runs + slots <= h->cap_runs;
    if ((st = ensure_run_workspace(h, runs, slots)) != FASTSV_OK) return fail(st);
    h->last_runs = runs;
    if (!fits) {
        // split now (one chunk), or again with room for every run
        for (int c = 0; c < C; ++c)
            if ((st = launch_chunk_split<RP>(h, pipelined ? B : one, c, s)) != FASTSV_OK) return fail(st);
    }
    FSV_CUDA(h, cudaStreamWaitEvent(s, h->side_ev[1], 0));  // the first iteration's hooks are done
    k_setup_blocks<<<1, 256, 0, s>>>(h->d_ctx, h->d_clay, C, B.nb, h->d_colB, h->d_rowsB, h->d_endsB, tile);
    k_scan_tiles<<<1, 1024, 0, s>>>(h->d_ctx);
    k_partition<int32_t><<<setup_grid(h), 256, 0, s>>>(h->d_ctx);
    h->pending_fixed_launches += 3;
    FSV_CUDA(h, cudaGetLastError());
    return FASTSV_OK;
}

static fastsv_status solve_single(fastsv_ctx* h, int64_t n, int64_t m, const void* rp, const int32_t* ci,
                                  int32_t* labels, cudaStream_t s, const int32_t* ci_host = nullptr) {
    const int rp64 = h->opt.rowptr_bits == 64;
    const int items = k2_items(h);
    // the ablation variants sv1..sv4 and the asynchronous mode run unblocked
    // and without sparse iterations
    const int variant = (h->opt.variant >= 1 && h->opt.variant <= 4) ? h->opt.variant : 0;
    const bool async = h->opt.mode == FASTSV_MODE_ASYNC;
    const bool plain = variant == 0 && !async;
    const int64_t tile = async ? (int64_t)ASYNC_THREADS * ASYNC_ITEMS : k2_tile(h);
    const int nb = (m > 0 && plain) ? choose_col_blocks(h, n, m) : 1;
    int shift = 0;
    while (shift < 31 && ((int64_t)nb << shift) < n) ++shift;
    const int nb_eff = nb > 1 ? (int)((n + (1ll << shift) - 1) >> shift) : 1;
    // a blocked solve partitions the graph itself for the first iteration and
    // the block copy first (BUILD_TILE items per tile)
    const int64_t tile0 = nb_eff > 1 ? (int64_t)BUILD_TILE : tile;
    const int64_t t2 = m > 0 ? (n + m + tile0 - 1) / tile0 : 0;
    // the blocks' tiles: every run holds at least one entry, so runs <= m;
    // one segment per block and chunk of the copy
    const int64_t bsegs = nb_eff > 1 ? (int64_t)nb_eff * FEED_CHUNKS : 0;
    const int64_t t2b = nb_eff > 1 ? (2 * m) / tile + 2 * (bsegs + 1) : 0;
    const int64_t t3 = (n + K3_TILE - 1) / K3_TILE;
    if (t2 > INT32_MAX || t2b > INT32_MAX || t3 > INT32_MAX) return FASTSV_ERR_UNSUPPORTED;
    fastsv_status st = ensure_workspace(h, n, t2 > t2b ? t2 : t2b, t3, 1 + bsegs);
    if (st != FASTSV_OK) return st;
    if (nb_eff > 1 && (st = ensure_block_workspace(h, nb_eff, t2, m)) != FASTSV_OK) return st;
    // col_idx still in host memory: a blocked solve without validation copies
    // it chunk by chunk under its first iteration; any other copies it now
    HostFeed feed{ci_host, const_cast<int32_t*>(ci)};
    const bool fed = ci_host && m > 0 && nb_eff > 1 && !h->opt.validate;
    if (ci_host && m > 0 && !fed)
        FSV_CUDA(h, cudaMemcpyAsync(const_cast<int32_t*>(ci), ci_host, (size_t)m * 4, cudaMemcpyHostToDevice, s));
    h->pending_fixed_launches = 0;
    h->ms_k2 = h->ms_k3 = h->ms_push = h->ms_hook = 0.f;
    h->dense_iters = 0;
    h->timed_iters = 0;
    h->last_col_blocks = nb_eff;
    FSV_CUDA(h, cudaEventRecord(h->ev_start, s));
    SingleParams prm;
    prm.rp = rp;
    prm.ci = ci;
    prm.f = labels;
    prm.p = h->d_p;
    prm.gf = variant == 1 ? h->d_p : h->d_gf;  // sv1's SpMV gathers parents, not grandparents
    prm.mngf = h->d_mngf;
    prm.frontier = h->d_frontier;
    prm.sparse_div = (plain && h->opt.sparse_div > 0) ? h->opt.sparse_div : 0;
    prm.n = n;
    prm.m = m;
    prm.k2_tile = (int32_t)tile0;
    prm.max_iters = h->opt.max_iters;
    prm.loop_limit = h->opt.max_iters + 1;
    WsPtrs ws{h->d_segs, h->d_k2_seg, h->d_k2_row, h->d_k3_seg};
    k_setup_single<<<1, 1, 0, s>>>(h->d_ctx, prm, ws);
    if (rp64)
        k_partition<int64_t><<<setup_grid(h), 256, 0, s>>>(h->d_ctx);
    else
        k_partition<int32_t><<<setup_grid(h), 256, 0, s>>>(h->d_ctx);
    h->pending_fixed_launches += 2;
    FSV_CUDA(h, cudaGetLastError());
    if ((st = run_validation(h, rp64, s)) != FASTSV_OK) return st;
    int loop_rp64 = rp64;
    if (nb_eff > 1) {
        // The graph's first iteration needs no gathers (gf is still the
        // identity), so it gains nothing from column blocks: it runs on the
        // original CSR, over the build's tiles (BUILD_TILE items), before the
        // block copy.  Fed from host memory, and with runs' arrays from an
        // earlier call, every chunk is copied into the blocks as soon as its
        // entries are in (checked, and redone if the runs did not fit).
        k_init_state<<<setup_grid(h), 256, 0, s>>>(h->d_ctx);
        h->pending_fixed_launches += 1;
        const bool pipelined = fed && h->cap_runs > 0;
        BlockBuild B{nb_eff, shift, FEED_CHUNKS, t2, m, fed ? h->d_feed_tiles : nullptr};
        if (fed && (st = ensure_feed(h)) != FASTSV_OK) return st;
        B.range = fed ? h->d_feed_tiles : nullptr;
        st = rp64 ? first_iteration_unblocked<int64_t>(h, B, fed ? &feed : nullptr, pipelined, s)
                  : first_iteration_unblocked<int32_t>(h, B, fed ? &feed : nullptr, pipelined, s);
        if (st != FASTSV_OK) return st;
        // split the entries into column blocks of compressed rows
        st = rp64 ? build_blocks<int64_t>(h, B, pipelined, (int32_t)tile, s)
                  : build_blocks<int32_t>(h, B, pipelined, (int32_t)tile, s);
        if (st != FASTSV_OK) return st;
        loop_rp64 = 0;
    } else {
        k_init_state<<<setup_grid(h), 256, 0, s>>>(h->d_ctx);
        h->pending_fixed_launches += 1;
    }
    if (variant == 1) {
        kv_iota<<<setup_grid(h), 256, 0, s>>>(h->d_gf, n);  // grandparents for the root test
        h->pending_fixed_launches += 1;
    }
    FSV_CUDA(h, cudaGetLastError());
    FSV_CUDA(h, cudaEventRecord(h->ev_setup, s));
    h->loop_limit_host = prm.loop_limit;
    if (variant)
        st = run_variant_loop(h, h->d_ctx, rp64, items, variant, n, labels, s);
    else if (async)
        st = run_async_loop(h, h->d_ctx, rp64, s);
    else
        st = run_loop(h, h->d_ctx, rp64, loop_rp64, items, nb_eff > 1 ? nb_eff : 0, s);
    if (st != FASTSV_OK) return st;
    return finish_call(h, s, nullptr, n, m, true);
}

}  // namespace fsv

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

void fastsv_default_options(fastsv_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->rowptr_bits = 64;
    o->mode = FASTSV_MODE_SYNC;
    o->max_iters = 4096;
    o->validate = 0;
    o->use_graph = 1;
    o->k2_items = 8;
    o->grid_ctas_per_sm = 0;
    o->timing = 1;
    o->fail_alloc_after = 0;
    o->col_blocks = 0;
    o->k2_threads = 256;
    o->sparse_div = 2;
    o->col_block_mib = 64;
    o->tune_cache = nullptr;
}

const char* fastsv_status_string(fastsv_status s) {
    switch (s) {
        case FASTSV_OK: return "FASTSV_OK";
        case FASTSV_ERR_INVALID_ARG: return "FASTSV_ERR_INVALID_ARG";
        case FASTSV_ERR_OOM: return "FASTSV_ERR_OOM";
        case FASTSV_ERR_CUDA: return "FASTSV_ERR_CUDA";
        case FASTSV_ERR_MAX_ITERS: return "FASTSV_ERR_MAX_ITERS";
        case FASTSV_ERR_TIMEOUT: return "FASTSV_ERR_TIMEOUT";
        case FASTSV_ERR_UNSUPPORTED: return "FASTSV_ERR_UNSUPPORTED";
        case FASTSV_ERR_INVALID_GRAPH: return "FASTSV_ERR_INVALID_GRAPH";
        case FASTSV_ERR_FULL: return "FASTSV_ERR_FULL";
    }
    return "FASTSV_UNKNOWN";
}

fastsv_status fastsv_create(fastsv_t* out, const fastsv_options* opt) {
    if (!out) return FASTSV_ERR_INVALID_ARG;
    *out = nullptr;
    fastsv_options o;
    if (opt)
        o = *opt;
    else
        fastsv_default_options(&o);
    if (o.rowptr_bits != 32 && o.rowptr_bits != 64) return FASTSV_ERR_INVALID_ARG;
    if (o.mode != FASTSV_MODE_SYNC && o.mode != FASTSV_MODE_ASYNC) return FASTSV_ERR_INVALID_ARG;
    if (o.max_iters < 1 || o.max_iters > (1 << 30)) return FASTSV_ERR_INVALID_ARG;
    if (o.validate < 0 || o.validate > 2) return FASTSV_ERR_INVALID_ARG;
    if (o.variant < 0 || o.variant > 5) return FASTSV_ERR_INVALID_ARG;
    if (o.sparse_div < 0 || o.batch_sparse_div < 0) return FASTSV_ERR_INVALID_ARG;
    if (o.mode == FASTSV_MODE_ASYNC && o.variant >= 1 && o.variant <= 4) return FASTSV_ERR_INVALID_ARG;
    fastsv_ctx* h = new fastsv_ctx();
    if (o.tune_cache) {
        if (tune_load(h, o.tune_cache) != FASTSV_OK) {
            delete h;
            return FASTSV_ERR_INVALID_ARG;
        }
        o.tune_cache = nullptr;  // the path is not kept
    }
    h->opt = o;
    h->base_opt = o;
    fastsv_status st = FASTSV_OK;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) {
        int l2 = 0;
        e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, h->device);
        h->l2_bytes = l2;
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->d_ctx, sizeof(Ctx));
    if (e == cudaSuccess) e = cudaMemset(h->d_ctx, 0, sizeof(Ctx));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_sum, sizeof(Summary));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_scalar, 256);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_start);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_setup);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev_end);
    if (e != cudaSuccess) {
        st = cuda_fail(h, e);
        fastsv_destroy(h);
        return st;
    }
    memset(h->h_sum, 0, sizeof(Summary));
    *out = h;
    return FASTSV_OK;
}

fastsv_status fastsv_destroy(fastsv_t h) {
    if (!h) return FASTSV_ERR_INVALID_ARG;
    if (h->pending && h->ev_end) cudaEventSynchronize(h->ev_end);
    pool_release(h);
    for (auto& kv : h->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    dev_free((void**)&h->d_ctx);
    dev_free((void**)&h->d_segs);
    dev_free((void**)&h->d_k2_seg);
    dev_free((void**)&h->d_k2_row);
    dev_free((void**)&h->d_k3_seg);
    dev_free((void**)&h->d_p);
    dev_free((void**)&h->d_gf);
    dev_free((void**)&h->d_mngf);
    dev_free((void**)&h->d_frontier);
    dev_free((void**)&h->d_counts);
    dev_free((void**)&h->d_sums);
    dev_free((void**)&h->d_colB);
    dev_free((void**)&h->d_rowsB);
    dev_free((void**)&h->d_endsB);
    dev_free((void**)&h->d_build_scalars);
    dev_free((void**)&h->d_clay);
    dev_free((void**)&h->d_ctot);
    dev_free((void**)&h->d_feed_tiles);
    if (h->feed_stream) cudaStreamDestroy(h->feed_stream);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    for (cudaEvent_t& ev : h->side_ev)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t& ev : h->feed_ev)
        if (ev) cudaEventDestroy(ev);
    dev_free(&h->d_rp_copy);
    dev_free((void**)&h->d_ci_copy);
    dev_free((void**)&h->d_lab_copy);
    if (h->h_sum) cudaFreeHost(h->h_sum);
    if (h->h_scalar) cudaFreeHost(h->h_scalar);
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->ev_setup) cudaEventDestroy(h->ev_setup);
    if (h->ev_end) cudaEventDestroy(h->ev_end);
    delete h;
    return FASTSV_OK;
}

static void record_empty_call(fastsv_ctx* h, int64_t n, int64_t m) {
    h->pending = false;
    h->last_status = FASTSV_OK;
    h->last_n = n;
    h->last_m = m;
    memset(h->h_sum, 0, sizeof(Summary));
    h->h_sum->converged = 1;
}

fastsv_status fastsv_cc(fastsv_t h, int64_t n, const void* row_ptr, const int32_t* col_idx, int32_t* labels_out,
                        void* stream) {
    if (!h || n < 0 || n > (int64_t)INT32_MAX) return FASTSV_ERR_INVALID_ARG;
    if (n == 0) {
        record_empty_call(h, 0, 0);
        return FASTSV_OK;
    }
    if (!row_ptr || !labels_out) return FASTSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    order_after_previous(h, s);
    const int w = h->opt.rowptr_bits / 8;
    FSV_CUDA(h, cudaMemcpyAsync(h->h_scalar, (const char*)row_ptr + (size_t)n * w, (size_t)w,
                                cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaStreamSynchronize(s));
    int64_t m = w == 8 ? *(int64_t*)h->h_scalar : (int64_t) * (int32_t*)h->h_scalar;
    if (m < 0) return FASTSV_ERR_INVALID_GRAPH;
    if (m > 0 && !col_idx) return FASTSV_ERR_INVALID_ARG;
    tune_apply(h, TUNE_SINGLE, n, m, 1, h->base_opt.rowptr_bits);
    return solve_single(h, n, m, row_ptr, col_idx, labels_out, s);
}

static fastsv_status ensure_copy(fastsv_ctx* h, void** buf, size_t* cap, size_t bytes) {
    if (bytes <= *cap && *buf) return FASTSV_OK;
    dev_free(buf);
    *cap = 0;
    fastsv_status st = dev_alloc(h, buf, bytes);
    if (st == FASTSV_OK) *cap = bytes;
    return st;
}

fastsv_status fastsv_get_stats(fastsv_t h, fastsv_stats* out);

fastsv_status fastsv_cc_host(fastsv_t h, int64_t n, const void* row_ptr_host, const int32_t* col_idx_host,
                             int32_t* labels_host, void* stream) {
    if (!h || n < 0 || n > (int64_t)INT32_MAX) return FASTSV_ERR_INVALID_ARG;
    if (n == 0) {
        record_empty_call(h, 0, 0);
        return FASTSV_OK;
    }
    if (!row_ptr_host || !labels_host) return FASTSV_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    order_after_previous(h, s);
    const int w = h->opt.rowptr_bits / 8;
    int64_t m = w == 8 ? ((const int64_t*)row_ptr_host)[n] : (int64_t)((const int32_t*)row_ptr_host)[n];
    if (m < 0) return FASTSV_ERR_INVALID_GRAPH;
    if (m > 0 && !col_idx_host) return FASTSV_ERR_INVALID_ARG;
    tune_apply(h, TUNE_SINGLE, n, m, 1, h->base_opt.rowptr_bits);
    fastsv_status st;
    if ((st = ensure_copy(h, &h->d_rp_copy, &h->cap_rp_copy, (size_t)(n + 1) * w)) != FASTSV_OK) return st;
    if ((st = ensure_copy(h, (void**)&h->d_ci_copy, &h->cap_ci_copy, (size_t)(m > 0 ? m : 1) * 4)) != FASTSV_OK)
        return st;
    if ((st = ensure_copy(h, (void**)&h->d_lab_copy, &h->cap_lab_copy, (size_t)n * 4)) != FASTSV_OK) return st;
    FSV_CUDA(h, cudaMemcpyAsync(h->d_rp_copy, row_ptr_host, (size_t)(n + 1) * w, cudaMemcpyHostToDevice, s));
    // col_idx is copied by the solve: for a column-blocked graph in chunks
    // that overlap its first iteration
    if ((st = solve_single(h, n, m, h->d_rp_copy, h->d_ci_copy, h->d_lab_copy, s, m > 0 ? col_idx_host : nullptr)) !=
        FASTSV_OK)
        return st;
    FSV_CUDA(h, cudaMemcpyAsync(labels_host, h->d_lab_copy, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaStreamSynchronize(s));
    fastsv_stats tmp;
    return fastsv_get_stats(h, &tmp);
}

fastsv_status fastsv_cc_batched(fastsv_t h, int32_t G, const int64_t* vtx_off, const int64_t* edge_off,
                                const int32_t* row_ptr, const int32_t* col_idx, int32_t* labels_out,
                                int32_t* iters_out, void* stream) {
    if (!h || G < 0) return FASTSV_ERR_INVALID_ARG;
    if (G == 0) {
        record_empty_call(h, 0, 0);
        return FASTSV_OK;
    }
    if (!vtx_off || !edge_off || !row_ptr || !labels_out) return FASTSV_ERR_INVALID_ARG;
    if (h->opt.mode != FASTSV_MODE_SYNC || (h->opt.variant >= 1 && h->opt.variant <= 4))
        return FASTSV_ERR_UNSUPPORTED;  // the ablation and the asynchronous mode are single-graph only
    cudaStream_t s = (cudaStream_t)stream;
    order_after_previous(h, s);
    FSV_CUDA(h, cudaMemcpyAsync(h->h_scalar, vtx_off + G, 8, cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaMemcpyAsync(h->h_scalar + 1, edge_off + G, 8, cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaStreamSynchronize(s));
    const int64_t N = h->h_scalar[0], M = h->h_scalar[1];
    if (N < 0 || M < 0) return FASTSV_ERR_INVALID_GRAPH;
    if (M > 0 && !col_idx) return FASTSV_ERR_INVALID_ARG;
    tune_apply(h, TUNE_BATCHED, N, M, G, 32);
    const int items = k2_items(h);
    const int64_t tile = k2_tile(h);
    const int64_t t2 = (N + M) / tile + G + 1;
    const int64_t t3 = N / K3_TILE + G + 1;
    if (t2 > INT32_MAX || t3 > INT32_MAX) return FASTSV_ERR_UNSUPPORTED;
    fastsv_status st = ensure_workspace(h, N > 0 ? N : 1, t2, t3, G);
    if (st != FASTSV_OK) return st;
    h->pending_fixed_launches = 0;
    h->ms_k2 = h->ms_k3 = h->ms_push = h->ms_hook = 0.f;
    h->dense_iters = 0;
    h->timed_iters = 0;
    FSV_CUDA(h, cudaEventRecord(h->ev_start, s));
    BatchParams prm;
    prm.G = G;
    prm.vtx_off = vtx_off;
    prm.edge_off = edge_off;
    prm.row_ptr = row_ptr;
    prm.col_idx = col_idx;
    prm.labels = labels_out;
    prm.p = h->d_p;
    prm.gf = h->d_gf;
    prm.mngf = h->d_mngf;
    prm.frontier = h->d_frontier;
    prm.frontier_cap = N;
    prm.sparse_div = h->opt.batch_sparse_div > 0 ? h->opt.batch_sparse_div : 0;
    prm.k2_tile = (int32_t)tile;
    prm.max_iters = h->opt.max_iters;
    prm.loop_limit = h->opt.max_iters + 1;
    WsPtrs ws{h->d_segs, h->d_k2_seg, h->d_k2_row, h->d_k3_seg};
    int gs = (G + 255) / 256;
    if (gs > setup_grid(h)) gs = setup_grid(h);
    k_setup_batched<<<gs, 256, 0, s>>>(h->d_ctx, prm, ws);
    k_scan_tiles<<<1, 1024, 0, s>>>(h->d_ctx);
    k_partition<int32_t><<<setup_grid(h), 256, 0, s>>>(h->d_ctx);
    k_init_state<<<setup_grid(h), 256, 0, s>>>(h->d_ctx);
    h->pending_fixed_launches += 4;
    FSV_CUDA(h, cudaGetLastError());
    if ((st = run_validation(h, 0, s)) != FASTSV_OK) return st;
    FSV_CUDA(h, cudaEventRecord(h->ev_setup, s));
    if (N > 0) {
        h->loop_limit_host = prm.loop_limit;
        if ((st = run_loop(h, h->d_ctx, 0, 0, items, 0, s)) != FASTSV_OK) return st;
    } else {
        h->pending_loop_kernels = 0;
    }
    return finish_call(h, s, iters_out, N, M, false);
}

fastsv_status fastsv_get_stats(fastsv_t h, fastsv_stats* out) {
    if (!h || !out) return FASTSV_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    float total = 0.f, setup = 0.f;
    if (h->pending) {
        cudaError_t e = cudaEventSynchronize(h->ev_end);
        if (e != cudaSuccess) {
            h->pending = false;
            return cuda_fail(h, e);
        }
        h->pending = false;
        const Summary& S = *h->h_sum;
        h->launches_loop_dev = (int64_t)S.loop_kernels;
        int st = FASTSV_OK;
        if (S.status & (DEV_ERR_BAD_ROWPTR | DEV_ERR_BAD_COLIDX | DEV_ERR_ASYMMETRIC))
            st = FASTSV_ERR_INVALID_GRAPH;
        else if (S.status & DEV_ERR_MAX_ITERS)
            st = FASTSV_ERR_MAX_ITERS;
        h->last_status = st;
        if (h->opt.timing) {
            cudaEventElapsedTime(&total, h->ev_start, h->ev_end);
            cudaEventElapsedTime(&setup, h->ev_start, h->ev_setup);
        }
        h->h_sum->iterations = S.iterations;  // keep for repeated queries
        out->ms_total = total;
        out->ms_setup = setup;
        h->ms_total_cache = total;
        h->ms_setup_cache = setup;
    } else {
        out->ms_total = h->ms_total_cache;
        out->ms_setup = h->ms_setup_cache;
    }
    const Summary& S = *h->h_sum;
    out->n = h->last_n;
    out->m = h->last_m;
    out->iterations = S.iterations;
    out->status = h->last_status;
    out->converged = S.converged;
    out->ms_k2 = h->ms_k2;
    out->ms_k3 = h->ms_k3;
    out->ms_push = h->ms_push;
    out->ms_hook = h->ms_hook;
    out->sparse_iters = S.sparse_iters;
    out->dense_iters = (int32_t)(S.iterations - S.sparse_iters);
    out->timed_iters = h->opt.use_graph ? 0 : h->timed_iters;
    out->timed_dense_iters = h->opt.use_graph ? 0 : h->dense_iters;
    int len = (int)(S.iterations < TRACE_LEN ? S.iterations : TRACE_LEN);
    out->trace_len = h->single ? len : 0;
    out->col_blocks = h->single ? h->last_col_blocks : 1;
    for (int i = 0; i < out->trace_len; ++i) out->changed_per_iter[i] = (int64_t)S.trace[i];
    out->block_runs = h->single && h->last_col_blocks > 1 ? h->last_runs : 0;
    out->tuned = h->last_tuned;
    return (fastsv_status)h->last_status;
}

int32_t fastsv_last_cuda_error(fastsv_t h) { return h ? h->last_cuda_error : 0; }

// the layouts the Python binding mirrors (its tests pin the same sizes)
static_assert(sizeof(fastsv_options) == 72, "fastsv_options layout");
static_assert(sizeof(fastsv_stats) == 608, "fastsv_stats layout");

int64_t fastsv_kernel_launches(fastsv_t h) { return h ? h->launches + h->launches_loop_dev : 0; }

}  // extern "C"

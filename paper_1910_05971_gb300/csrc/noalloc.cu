// noalloc.cu -- fastsv_cc_noalloc: connected components without any device
// allocation by the library.
//
// Who needs this: callers that must not allocate device memory while they
// run -- a host framework that has reserved all device memory in its own
// pool (cudaMalloc would fail or fragment that pool), latency-critical loops
// that cannot afford cudaMalloc/cudaFree (both can synchronise the whole
// device), and code that is not allowed to call an allocator at all.  They
// pass their input graph and output buffer; everything else the solve needs
// lives in one fixed scratch array compiled into this library.
//
// The scratch is a file-scope __device__ array of FASTSV_NOALLOC_MAX_VERTICES
// vertices' worth of state (two int32 vectors) plus a counter; every GPU
// that loads the library keeps it until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it.  All calls on a device share the array: calls that overlap
// on the GPU race on it, and each call re-initialises what it reads.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "../../include/fastsv.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;

// p (snapshot of the parent vector), gf (grandparents), and one changed counter
struct NaScratch {
    int32_t p[FASTSV_NOALLOC_MAX_VERTICES];
    int32_t gf[FASTSV_NOALLOC_MAX_VERTICES];
    unsigned long long changed;
};

__device__ __align__(256) NaScratch na_scratch;

std::mutex na_mutex;
NaScratch* na_ptr[NA_MAX_DEVICES] = {};

// address of the scratch on the current device (looked up once per device)
fastsv_status na_scratch_ptr(NaScratch** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        (void)cudaGetLastError();
        return FASTSV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return FASTSV_ERR_CUDA;
        }
        na_ptr[dev] = (NaScratch*)p;
    }
    *out = na_ptr[dev];
    return FASTSV_OK;
}

// f = p = gf = identity (Algorithm 2 initialisation)
__global__ void na_init(NaScratch* s, int32_t* f, int32_t n) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        f[v] = v;
        s->p[v] = v;
        s->gf[v] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) s->changed = 0;
}

// one warp per row: mngf = min of gf over the row's neighbours, then the
// stochastic hook f[p[u]] <-min mngf, and the aggressive hook and shortcut
// f[u] <-min min(mngf, gf[u]) (atomic mins of values read from p and gf, so
// the result does not depend on scheduling)
__global__ void na_hook(NaScratch* s, const int32_t* rp, const int32_t* ci, int32_t* f, int32_t n) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int32_t b = rp[u], e = rp[u + 1];
        int32_t mn = INT_MAX;
        for (int32_t k = b + lane; k < e; k += 32) {
            const int32_t v = ci[k];
            if ((uint32_t)v < (uint32_t)n) mn = min(mn, s->gf[v]);
        }
        mn = (int32_t)__reduce_min_sync(0xffffffffu, (unsigned)mn);
        if (lane == 0 && mn != INT_MAX) {
            const int32_t g = s->gf[u], pu = s->p[u];
            if (mn < g) atomicMin(f + pu, mn);
            const int32_t m2 = mn < g ? mn : g;
            if (m2 < pu) atomicMin(f + u, m2);
        }
    }
}

// gf' = f[f]; count changes (termination test of Section 3.4); p = f
__global__ void na_grand(NaScratch* s, const int32_t* f, int32_t n) {
    unsigned c = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int32_t fv = f[v];
        const int32_t g = f[fv];
        if (g != s->gf[v]) {
            s->gf[v] = g;
            ++c;
        }
        s->p[v] = fv;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s->changed, (unsigned long long)c);
}

}  // namespace

extern "C" fastsv_status fastsv_cc_noalloc(int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                           int32_t* labels_out, int32_t max_iters, int32_t* iterations_out,
                                           void* stream) {
    if (iterations_out) *iterations_out = 0;
    if (n < 0 || max_iters < 1) return FASTSV_ERR_INVALID_ARG;
    if (n > FASTSV_NOALLOC_MAX_VERTICES) return FASTSV_ERR_UNSUPPORTED;
    if (n == 0) return FASTSV_OK;
    if (!row_ptr || !labels_out) return FASTSV_ERR_INVALID_ARG;
    NaScratch* s = nullptr;
    fastsv_status st = na_scratch_ptr(&s);
    if (st != FASTSV_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const int32_t nn = (int32_t)n;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return FASTSV_ERR_CUDA;
    }
    const int grid_v = (int)((n + NA_THREADS - 1) / NA_THREADS) < sms * 8 ? (int)((n + NA_THREADS - 1) / NA_THREADS)
                                                                          : sms * 8;
    const int grid_w = sms * 8;
    na_init<<<grid_v, NA_THREADS, 0, cs>>>(s, labels_out, nn);
    unsigned long long changed = 0;
    int32_t it = 0;
    cudaError_t e = cudaGetLastError();
    while (e == cudaSuccess) {
        // the counter keeps the previous iteration's (or call's) value: clear it
        e = cudaMemsetAsync(&s->changed, 0, sizeof(unsigned long long), cs);
        if (e != cudaSuccess) break;
        if (col_idx) na_hook<<<grid_w, NA_THREADS, 0, cs>>>(s, row_ptr, col_idx, labels_out, nn);
        na_grand<<<grid_v, NA_THREADS, 0, cs>>>(s, labels_out, nn);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&changed, &s->changed, sizeof(changed), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) break;
        ++it;
        if (changed == 0 || it >= max_iters) break;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return FASTSV_ERR_CUDA;
    }
    if (iterations_out) *iterations_out = it;
    return changed != 0 ? FASTSV_ERR_MAX_ITERS : FASTSV_OK;
}

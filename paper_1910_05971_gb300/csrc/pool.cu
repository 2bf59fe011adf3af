// pool.cu -- serving pool: continuous batching of independent CC queries.
//
// A pool owns one HBM arena (the admission budget) and a segment table with
// one fixed entry per slot.  Admitting a graph copies its CSR from host
// memory into an arena region and writes its slot's entry; fastsv_pool_step
// rebuilds the merge-path tile lists over the active slots and runs the same
// device-side FastSV loop as the batched solve (Algorithm 2 with per-graph
// early termination, Section 3.4) for a bounded number of iterations.  A
// slot's state (f, p, gf, iteration count) stays resident between steps, so
// graphs admitted later join the running batch at an iteration boundary and
// every graph follows exactly the iteration sequence it has alone.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "fastsv_internal.h"

namespace fsv {

constexpr int ADMIT_MAX = 48;
constexpr size_t ALIGN = 256;

struct AdmitDesc {
    const int32_t* rp;
    const int32_t* ci;
    int32_t* f;
    int32_t* p;
    int32_t* gf;
    int32_t* mngf;
    int64_t n, m;
    int32_t slot;
    int32_t iters0;  // iterations already run (a graph restored from a checkpoint), else 0
};

struct AdmitBatch {
    AdmitDesc d[ADMIT_MAX];
    int32_t count;
    int32_t num_slots;
    int32_t k2_tile;
    int32_t max_iters;
    int32_t loop_limit;
    int32_t pad;
};

// writes the entries of newly admitted slots and the step's loop scalars
__global__ void k_pool_admit(Ctx* ctx, Seg* segs, int32_t* k2_seg, int32_t* k2_row, int32_t* k3_seg,
                             AdmitBatch b) {
    const int i = threadIdx.x;
    if (i < b.count) {
        const AdmitDesc& a = b.d[i];
        Seg s;
        s.rp = a.rp;
        s.ci = a.ci;
        s.f = a.f;
        s.p = a.p;
        s.gf = a.gf;
        s.n = a.n;
        s.m = a.m;
        s.k2_tile0 = 0;
        s.k3_tile0 = 0;
        s.k2_ntiles = (a.m > 0 && a.n > 0) ? (int32_t)((a.n + a.m + b.k2_tile - 1) / b.k2_tile) : 0;
        s.k3_ntiles = (int32_t)((a.n + K3_TILE - 1) / K3_TILE);
        s.active = a.n > 0;
        s.iters = a.iters0;  // > 0 keeps the restored f, p, gf (k_init_state skips the slot)
        s.status = 0;
        s.converged = a.n == 0;
        s.changed = 0;
        s.user = a.slot;
        s.leader = a.slot;
        s.mode = 0;  // a restored graph's mngf is not kept: its first step runs a full SpMV
        s.mngf = a.mngf;
        s.fr_deg = 0;
        s.rowmap = nullptr;
        segs[a.slot] = s;
    }
    if (i == 0) {
        ctx->segs = segs;
        ctx->k2_tile_seg = k2_seg;
        ctx->k2_tile_row = k2_row;
        ctx->k3_tile_seg = k3_seg;
        ctx->num_segs = b.num_slots;
        ctx->k2_tile = b.k2_tile;
        ctx->max_iters = b.max_iters;
        ctx->loop_limit = b.loop_limit;
        ctx->loop_iter = 0;
        ctx->k3_done = 0;
        ctx->val_status = 0;
    }
}

// start of a step: the device loop's iteration counter and cap, and the
// sparse-iteration state (pool-owned frontier; kinds of work of the first
// iteration from the resident graphs' modes)
__global__ void k_pool_begin(Ctx* ctx, int32_t loop_limit, int32_t* frontier, int64_t frontier_cap,
                             int32_t sparse_div) {
    __shared__ int s_dense, s_push;
    if (threadIdx.x == 0) s_dense = s_push = 0;
    __syncthreads();
    int dense = 0, push = 0;
    for (int i = threadIdx.x; i < ctx->num_segs; i += blockDim.x) {
        const Seg& S = ctx->segs[i];
        if (!S.active) continue;
        if (S.mode)
            push = 1;
        else
            dense = 1;
    }
    if (dense) s_dense = 1;
    if (push) s_push = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        ctx->loop_iter = 0;
        ctx->loop_limit = loop_limit;
        ctx->k3_done = 0;
        ctx->sparse_enabled = sparse_div > 0 && frontier != nullptr;
        ctx->sparse_div = sparse_div;
        ctx->blk_chunks = 1;
        ctx->frontier = frontier;
        ctx->frontier_cap = (unsigned int)(frontier_cap < 0x7fffffff ? frontier_cap : 0x7fffffff);
        ctx->mode = (s_dense ? MODE_DENSE : 0) | (s_push ? MODE_PUSH : 0);
    }
}

struct Slot {
    int state = 0;  // 0 free, 1 admitted (copies in flight), 2 iterating on the device
    cudaEvent_t copied = nullptr;  // recorded on the copy stream after the slot's copies
    int64_t n = 0, m = 0;
    size_t off = 0, bytes = 0;
    int32_t* labels_host = nullptr;
    int32_t iters0 = 0;  // iterations run before a restore
};

// host checkpoint of one graph at an iteration boundary: header, f[n], gf[n]
constexpr uint32_t CKPT_MAGIC = 0x46535643u;  // "FSVC"
constexpr uint32_t CKPT_VERSION = 1;
constexpr size_t CKPT_HEADER = 64;
struct CkptHeader {
    uint32_t magic, version;
    int64_t n, m;
    int32_t iters, status;
};
static_assert(sizeof(CkptHeader) <= CKPT_HEADER, "checkpoint header");

// offsets of the vectors inside a slot's region: rp, ci, f, p, gf, mngf
static size_t off_f(int64_t n, int64_t m);

struct Pool {
    Ctx* d_ctx = nullptr;
    Seg* d_segs = nullptr;
    Seg* h_segs = nullptr;  // pinned mirror of the segment table after each step
    int32_t* d_k2_seg = nullptr;
    int32_t* d_k2_row = nullptr;
    int32_t* d_k3_seg = nullptr;
    int32_t* d_frontier = nullptr;  // (slot, vertex) pairs of the last iteration's changed vertices
    int64_t frontier_cap = 0;       // pairs
    char* arena = nullptr;
    size_t budget = 0, used = 0;
    std::map<size_t, size_t> free_list;  // offset -> size, coalesced
    int max_slots = 0;
    std::vector<Slot> slots;
    std::vector<int> admitted;  // slots whose copies were enqueued since the last step
    cudaStream_t copy_stream = nullptr;  // admissions (host to device), may run during a step
    cudaStream_t out_stream = nullptr;   // harvests (labels to host)
    cudaEvent_t step_done = nullptr;
    cudaEvent_t ev_t[4] = {};  // step phases: start, copies landed, set-up done, loop done
    bool timed = false;        // the last step recorded ev_t
    bool stepped = false;
    bool dirty = false;
};

static size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// a slot back to free (its copy event is kept for the next graph)
static void slot_reset(Slot& S) {
    cudaEvent_t ev = S.copied;
    S = Slot();
    S.copied = ev;
}

static size_t region_bytes(int64_t n, int64_t m) {
    return align_up((size_t)(n + 1) * 4) + align_up((size_t)(m > 0 ? m : 1) * 4) + 4 * align_up((size_t)n * 4);
}
static size_t off_f(int64_t n, int64_t m) {
    return align_up((size_t)(n + 1) * 4) + align_up((size_t)(m > 0 ? m : 1) * 4);
}
static size_t off_p(int64_t n, int64_t m) { return off_f(n, m) + align_up((size_t)n * 4); }
static size_t off_gf(int64_t n, int64_t m) { return off_p(n, m) + align_up((size_t)n * 4); }

static bool arena_alloc(Pool* P, size_t bytes, size_t* off) {
    for (auto it = P->free_list.begin(); it != P->free_list.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            size_t rest = it->second - bytes;
            size_t start = it->first + bytes;
            P->free_list.erase(it);
            if (rest) P->free_list[start] = rest;
            P->used += bytes;
            return true;
        }
    }
    return false;
}

static void arena_free(Pool* P, size_t off, size_t bytes) {
    P->used -= bytes;
    auto it = P->free_list.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != P->free_list.end() && it->first + it->second == next->first) {
        it->second += next->second;
        P->free_list.erase(next);
    }
    if (it != P->free_list.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            P->free_list.erase(it);
        }
    }
}

void pool_release(fastsv_ctx* h) {
    Pool* P = h->pool;
    if (!P) return;
    if (P->step_done) cudaEventSynchronize(P->step_done);
    if (P->copy_stream) cudaStreamSynchronize(P->copy_stream);
    if (P->out_stream) cudaStreamSynchronize(P->out_stream);
    if (P->d_ctx) cudaFree(P->d_ctx);
    if (P->d_segs) cudaFree(P->d_segs);
    if (P->h_segs) cudaFreeHost(P->h_segs);
    if (P->d_k2_seg) cudaFree(P->d_k2_seg);
    if (P->d_k2_row) cudaFree(P->d_k2_row);
    if (P->d_k3_seg) cudaFree(P->d_k3_seg);
    if (P->d_frontier) cudaFree(P->d_frontier);
    if (P->arena) cudaFree(P->arena);
    if (P->copy_stream) cudaStreamDestroy(P->copy_stream);
    if (P->out_stream) cudaStreamDestroy(P->out_stream);
    if (P->step_done) cudaEventDestroy(P->step_done);
    for (cudaEvent_t& ev : P->ev_t)
        if (ev) cudaEventDestroy(ev);
    for (Slot& S : P->slots)
        if (S.copied) cudaEventDestroy(S.copied);
    delete P;
    h->pool = nullptr;
}

}  // namespace fsv

using namespace fsv;

extern "C" {

size_t fastsv_pool_bytes(int64_t n, int64_t m) {
    if (n < 0 || m < 0) return 0;
    return region_bytes(n, m);
}

fastsv_status fastsv_pool_create(fastsv_t h, size_t budget, int32_t max_slots) {
    if (!h || budget < ALIGN || max_slots < 1 || max_slots > (1 << 20)) return FASTSV_ERR_INVALID_ARG;
    if (h->pool) return FASTSV_ERR_INVALID_ARG;
    if (h->opt.mode != FASTSV_MODE_SYNC || (h->opt.variant >= 1 && h->opt.variant <= 4))
        return FASTSV_ERR_UNSUPPORTED;  // the pool runs the default iteration only
    Pool* P = new Pool();
    h->pool = P;
    P->budget = budget / ALIGN * ALIGN;
    P->max_slots = max_slots;
    P->slots.resize(max_slots);
    const int64_t tile = k2_tile(h);
    // every slot needs at least 4(n+m) bytes, so n + m <= budget / 4 over all slots
    const int64_t cap2 = (int64_t)(P->budget / 4) / tile + max_slots + 1;
    const int64_t cap3 = (int64_t)(P->budget / 16) / K3_TILE + max_slots + 1;
    // every resident vertex needs >= 20 bytes of the arena; a larger frontier
    // than 2^27 pairs (1 GiB) overflows into a full SpMV for one iteration
    const int64_t fcap = std::min<int64_t>((int64_t)(P->budget / 20) + 1, (int64_t)1 << 27);
    P->frontier_cap = fcap;
    fastsv_status st = FASTSV_OK;
    cudaError_t e = cudaSuccess;
    if ((st = dev_alloc(h, (void**)&P->d_ctx, sizeof(Ctx))) != FASTSV_OK ||
        (st = dev_alloc(h, (void**)&P->d_segs, sizeof(Seg) * (size_t)max_slots)) != FASTSV_OK ||
        (st = dev_alloc(h, (void**)&P->d_k2_seg, 4 * (size_t)cap2)) != FASTSV_OK ||
        (st = dev_alloc(h, (void**)&P->d_k2_row, 4 * (size_t)cap2)) != FASTSV_OK ||
        (st = dev_alloc(h, (void**)&P->d_k3_seg, 4 * (size_t)cap3)) != FASTSV_OK ||
        (st = dev_alloc(h, (void**)&P->d_frontier, 8 * (size_t)fcap)) != FASTSV_OK ||
        (st = dev_alloc(h, (void**)&P->arena, P->budget)) != FASTSV_OK) {
        pool_release(h);
        return st;
    }
    e = cudaMemset(P->d_ctx, 0, sizeof(Ctx));
    // Touch the whole arena once, now: measured on GB300, copies into pages
    // of a fresh allocation that were never written run at ~32 GB/s against
    // ~210 GB/s afterwards, which would throttle the first admissions into
    // every region.  Writing 120 GB this way takes about a second, once, at
    // pool creation (synchronised here, so that no step waits behind it).
    if (e == cudaSuccess) e = cudaMemset(P->arena, 0, P->budget);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemset(P->d_segs, 0, sizeof(Seg) * (size_t)max_slots);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&P->h_segs, sizeof(Seg) * (size_t)max_slots);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->out_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->step_done, cudaEventDisableTiming);
    for (int i = 0; i < 4 && e == cudaSuccess && h->opt.timing; ++i) e = cudaEventCreate(&P->ev_t[i]);
    for (int i = 0; i < max_slots && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&P->slots[i].copied, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        st = cuda_fail(h, e);
        pool_release(h);
        return st;
    }
    memset(P->h_segs, 0, sizeof(Seg) * (size_t)max_slots);
    P->free_list[0] = P->budget;
    return FASTSV_OK;
}

}  // extern "C"

namespace fsv {

// admit a graph: a slot, an arena region, the copies of its CSR (and, for a
// restore, of its checkpointed f -> f and p, gf -> gf) on the copy stream
static fastsv_status admit(fastsv_t h, int64_t n, const int32_t* rp, const int32_t* ci, int32_t* labels_host,
                           const unsigned char* ckpt, int32_t* slot_out) {
    if (!h || !h->pool || !slot_out || n < 0 || n > (int64_t)INT32_MAX) return FASTSV_ERR_INVALID_ARG;
    if (!rp || (n > 0 && !labels_host)) return FASTSV_ERR_INVALID_ARG;
    Pool* P = h->pool;
    *slot_out = -1;
    const int64_t m = rp[n];
    if (m < 0 || (m > 0 && !ci)) return FASTSV_ERR_INVALID_ARG;
    int32_t iters0 = 0;
    if (ckpt) {
        CkptHeader hd;
        memcpy(&hd, ckpt, sizeof(hd));
        if (hd.magic != CKPT_MAGIC || hd.version != CKPT_VERSION || hd.n != n || hd.m != m || hd.iters < 1)
            return FASTSV_ERR_INVALID_ARG;
        iters0 = hd.iters;
    }
    const size_t bytes = region_bytes(n, m);
    if (bytes > P->budget) return FASTSV_ERR_INVALID_ARG;  // can never fit
    int slot = -1;
    for (int s = 0; s < P->max_slots; ++s)
        if (P->slots[s].state == 0) {
            slot = s;
            break;
        }
    if (slot < 0) return FASTSV_ERR_FULL;
    size_t off = 0;
    if (!arena_alloc(P, bytes, &off)) return FASTSV_ERR_FULL;
    Slot& S = P->slots[slot];
    S.state = 1;
    S.n = n;
    S.m = m;
    S.off = off;
    S.bytes = bytes;
    S.labels_host = labels_host;
    S.iters0 = iters0;
    char* base = P->arena + off;
    cudaError_t e = cudaMemcpyAsync(base, rp, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, P->copy_stream);
    if (e == cudaSuccess && m > 0)
        e = cudaMemcpyAsync(base + align_up((size_t)(n + 1) * 4), ci, (size_t)m * 4, cudaMemcpyHostToDevice,
                            P->copy_stream);
    if (e == cudaSuccess && ckpt && n > 0) {
        const unsigned char* fh = ckpt + CKPT_HEADER;
        const unsigned char* gh = fh + (size_t)n * 4;
        e = cudaMemcpyAsync(base + off_f(n, m), fh, (size_t)n * 4, cudaMemcpyHostToDevice, P->copy_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + off_p(n, m), fh, (size_t)n * 4, cudaMemcpyHostToDevice, P->copy_stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + off_gf(n, m), gh, (size_t)n * 4, cudaMemcpyHostToDevice, P->copy_stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(S.copied, P->copy_stream);
    if (e != cudaSuccess) {
        arena_free(P, off, bytes);
        slot_reset(S);
        return cuda_fail(h, e);
    }
    P->admitted.push_back(slot);
    *slot_out = slot;
    return FASTSV_OK;
}

// the last step has finished: its device loop's kernels are counted
static fastsv_status settle_step(fastsv_t h, Pool* P) {
    if (!P->stepped) return FASTSV_OK;
    cudaError_t e = cudaEventSynchronize(P->step_done);
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (h->pool_loop_pending) {
        h->launches += (int64_t)h->pending_loop_kernels * *(int32_t*)(h->h_scalar + 2);
        h->pool_loop_pending = false;
    }
    return FASTSV_OK;
}

}  // namespace fsv

extern "C" {

fastsv_status fastsv_pool_add(fastsv_t h, int64_t n, const int32_t* rp, const int32_t* ci, int32_t* labels_host,
                              int32_t* slot_out) {
    return admit(h, n, rp, ci, labels_host, nullptr, slot_out);
}

size_t fastsv_pool_checkpoint_bytes(int64_t n) {
    if (n < 0) return 0;
    return CKPT_HEADER + 8 * (size_t)n;
}

fastsv_status fastsv_pool_evict(fastsv_t h, int32_t slot, void* checkpoint_host) {
    if (!h || !h->pool || !checkpoint_host) return FASTSV_ERR_INVALID_ARG;
    Pool* P = h->pool;
    if (slot < 0 || slot >= P->max_slots || P->slots[slot].state != 2) return FASTSV_ERR_INVALID_ARG;
    fastsv_status st = settle_step(h, P);
    if (st != FASTSV_OK) return st;
    Slot& S = P->slots[slot];
    const Seg& D = P->h_segs[slot];
    if (!D.active || S.n == 0) return FASTSV_ERR_INVALID_ARG;  // finished: harvest it with fastsv_pool_poll
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = CKPT_MAGIC;
    hd.version = CKPT_VERSION;
    hd.n = S.n;
    hd.m = S.m;
    hd.iters = D.iters;
    hd.status = D.status;
    unsigned char* out = (unsigned char*)checkpoint_host;
    memset(out, 0, CKPT_HEADER);
    memcpy(out, &hd, sizeof(hd));
    const char* base = P->arena + S.off;
    cudaError_t e = cudaMemcpyAsync(out + CKPT_HEADER, base + off_f(S.n, S.m), (size_t)S.n * 4,
                                    cudaMemcpyDeviceToHost, P->copy_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + CKPT_HEADER + (size_t)S.n * 4, base + off_gf(S.n, S.m), (size_t)S.n * 4,
                            cudaMemcpyDeviceToHost, P->copy_stream);
    // the slot leaves the device loop: no later step may touch its region
    if (e == cudaSuccess) e = cudaMemsetAsync(&P->d_segs[slot].active, 0, sizeof(int32_t), P->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->copy_stream);
    if (e != cudaSuccess) return cuda_fail(h, e);
    P->h_segs[slot].active = 0;
    P->dirty = true;  // its tiles leave the lists at the next step
    arena_free(P, S.off, S.bytes);
    slot_reset(S);
    return FASTSV_OK;
}

fastsv_status fastsv_pool_restore(fastsv_t h, int64_t n, const int32_t* rp, const int32_t* ci, int32_t* labels_host,
                                  const void* checkpoint_host, int32_t* slot_out) {
    if (!checkpoint_host) return FASTSV_ERR_INVALID_ARG;
    return admit(h, n, rp, ci, labels_host, (const unsigned char*)checkpoint_host, slot_out);
}

fastsv_status fastsv_pool_step(fastsv_t h, int32_t iters, void* stream) {
    if (!h || !h->pool || iters < 1) return FASTSV_ERR_INVALID_ARG;
    Pool* P = h->pool;
    cudaStream_t s = (cudaStream_t)stream;
    h->opt = h->base_opt;  // pools run the handle's own options (no tuning-cache lookup)
    h->last_tuned = 0;
    const int items = k2_items(h);
    const int32_t tile = (int32_t)k2_tile(h);
    // the slot snapshot read below must be the previous step's final one
    if (P->stepped) FSV_CUDA(h, cudaEventSynchronize(P->step_done));
    const bool timed = P->ev_t[0] != nullptr;
    if (timed) FSV_CUDA(h, cudaEventRecord(P->ev_t[0], s));
    // graphs whose copies have landed join this step; the others keep
    // copying while it runs and join a later one.  If nothing would run,
    // the step waits for the first admitted graph's copies instead.
    std::vector<int> joining, later;
    for (int slot : P->admitted) {
        if (h->opt.pool_wait_copies) {
            FSV_CUDA(h, cudaStreamWaitEvent(s, P->slots[slot].copied, 0));
            joining.push_back(slot);
            continue;
        }
        const cudaError_t q = cudaEventQuery(P->slots[slot].copied);
        if (q == cudaSuccess)
            joining.push_back(slot);
        else if (q == cudaErrorNotReady)
            later.push_back(slot);
        else
            return cuda_fail(h, q);
    }
    bool resident = false;
    for (int i = 0; i < P->max_slots && !resident; ++i)
        resident = P->slots[i].state == 2 && P->h_segs[i].active;
    if (joining.empty() && !resident && !later.empty()) {
        joining.push_back(later.front());
        later.erase(later.begin());
        FSV_CUDA(h, cudaStreamWaitEvent(s, P->slots[joining[0]].copied, 0));
    }
    P->admitted = joining;
    size_t na = P->admitted.size();
    if (timed) FSV_CUDA(h, cudaEventRecord(P->ev_t[1], s));
    size_t done = 0;
    do {
        AdmitBatch b;
        memset(&b, 0, sizeof(b));
        b.num_slots = P->max_slots;
        b.k2_tile = tile;
        b.max_iters = h->opt.max_iters;
        b.loop_limit = iters;
        while (done < na && b.count < ADMIT_MAX) {
            int slot = P->admitted[done++];
            Slot& S = P->slots[slot];
            char* base = P->arena + S.off;
            AdmitDesc& a = b.d[b.count++];
            a.rp = (const int32_t*)base;
            size_t o = align_up((size_t)(S.n + 1) * 4);
            a.ci = (const int32_t*)(base + o);
            o += align_up((size_t)(S.m > 0 ? S.m : 1) * 4);
            a.f = (int32_t*)(base + o);
            o += align_up((size_t)S.n * 4);
            a.p = (int32_t*)(base + o);
            o += align_up((size_t)S.n * 4);
            a.gf = (int32_t*)(base + o);
            o += align_up((size_t)S.n * 4);
            a.mngf = (int32_t*)(base + o);
            a.n = S.n;
            a.m = S.m;
            a.slot = slot;
            a.iters0 = S.iters0;
            S.state = 2;
        }
        k_pool_admit<<<1, ADMIT_MAX, 0, s>>>(P->d_ctx, P->d_segs, P->d_k2_seg, P->d_k2_row, P->d_k3_seg, b);
        h->launches += 1;
        FSV_CUDA(h, cudaGetLastError());
    } while (done < na);
    if (na > 0) P->dirty = true;
    P->admitted = later;
    if (P->dirty) {
        fastsv_status st = rebuild_tiles(h, P->d_ctx, s);
        if (st != FASTSV_OK) return st;
        P->dirty = false;
    }
    // work remains if graphs were just admitted or the last step's snapshot
    // shows a resident slot still iterating
    bool any = na > 0 || resident;
    if (timed) FSV_CUDA(h, cudaEventRecord(P->ev_t[2], s));
    if (any) {
        h->loop_limit_host = iters;
        const bool graph = h->opt.use_graph != 0;
        // every step runs up to `iters` iterations, whether or not it admitted
        k_pool_begin<<<1, 256, 0, s>>>(P->d_ctx, iters, P->d_frontier, P->frontier_cap,
                                       h->opt.batch_sparse_div > 0 ? h->opt.batch_sparse_div : 0);
        h->launches += 1;
        FSV_CUDA(h, cudaGetLastError());
        fastsv_status st = run_loop(h, P->d_ctx, 0, 0, items, 0, s);
        if (st != FASTSV_OK) return st;
        if (graph) {
            // the loop's iteration count is read back with the segment table
            FSV_CUDA(h, cudaMemcpyAsync(h->h_scalar + 2, &P->d_ctx->loop_iter, sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, s));
        }
    }
    if (timed) FSV_CUDA(h, cudaEventRecord(P->ev_t[3], s));
    FSV_CUDA(h, cudaMemcpyAsync(P->h_segs, P->d_segs, sizeof(Seg) * (size_t)P->max_slots, cudaMemcpyDeviceToHost, s));
    FSV_CUDA(h, cudaEventRecord(P->step_done, s));
    P->stepped = true;
    P->timed = timed;
    h->pool_loop_pending = any && h->opt.use_graph;
    return FASTSV_OK;
}

fastsv_status fastsv_pool_poll(fastsv_t h, int32_t* done_slots, int32_t* done_iters, int32_t cap, int32_t* n_done,
                               int32_t* n_active) {
    if (!h || !h->pool || !n_done || cap < 0 || (cap > 0 && !done_slots)) return FASTSV_ERR_INVALID_ARG;
    Pool* P = h->pool;
    *n_done = 0;
    fastsv_status sst = settle_step(h, P);
    if (sst != FASTSV_OK) return sst;
    int nd = 0, act = 0;
    std::vector<int> harvested;
    for (int i = 0; i < P->max_slots; ++i) {
        Slot& S = P->slots[i];
        if (S.state != 2) {
            if (S.state == 1) ++act;
            continue;
        }
        const Seg& D = P->h_segs[i];
        const bool finished = P->stepped && !D.active && (D.iters > 0 || S.n == 0);
        if (!finished) {
            ++act;
            continue;
        }
        if (nd >= cap) {
            ++act;
            continue;
        }
        if (S.n > 0) {
            size_t o = align_up((size_t)(S.n + 1) * 4) + align_up((size_t)(S.m > 0 ? S.m : 1) * 4);
            cudaError_t e = cudaMemcpyAsync(S.labels_host, P->arena + S.off + o, (size_t)S.n * 4,
                                            cudaMemcpyDeviceToHost, P->out_stream);
            if (e != cudaSuccess) return cuda_fail(h, e);
        }
        done_slots[nd] = i;
        if (done_iters) done_iters[nd] = (D.status & DEV_ERR_MAX_ITERS) ? -D.iters : D.iters;
        ++nd;
        harvested.push_back(i);
    }
    if (!harvested.empty()) {
        // admission copies of graphs added since the last step may still be
        // running on the copy stream: harvests wait only for their own copies
        cudaError_t e = cudaStreamSynchronize(P->out_stream);
        if (e != cudaSuccess) return cuda_fail(h, e);
        for (int i : harvested) {
            Slot& S = P->slots[i];
            arena_free(P, S.off, S.bytes);
            slot_reset(S);
        }
        P->dirty = true;  // the next step's tile lists leave the finished graphs out
    }
    *n_done = nd;
    if (n_active) *n_active = act;
    return FASTSV_OK;
}

fastsv_status fastsv_pool_step_times(fastsv_t h, float* ms_out) {
    if (!h || !h->pool || !ms_out) return FASTSV_ERR_INVALID_ARG;
    Pool* P = h->pool;
    ms_out[0] = ms_out[1] = ms_out[2] = 0.f;
    if (!P->stepped || !P->timed) return FASTSV_OK;
    fastsv_status st = settle_step(h, P);
    if (st != FASTSV_OK) return st;
    for (int i = 0; i < 3; ++i)
        if (cudaEventElapsedTime(&ms_out[i], P->ev_t[i], P->ev_t[i + 1]) != cudaSuccess) {
            (void)cudaGetLastError();
            ms_out[i] = 0.f;
        }
    return FASTSV_OK;
}

fastsv_status fastsv_pool_usage(fastsv_t h, int32_t* slots_used, size_t* bytes_used) {
    if (!h || !h->pool) return FASTSV_ERR_INVALID_ARG;
    Pool* P = h->pool;
    int u = 0;
    for (const Slot& S : P->slots) u += S.state != 0;
    if (slots_used) *slots_used = u;
    if (bytes_used) *bytes_used = P->used;
    return FASTSV_OK;
}

}  // extern "C"

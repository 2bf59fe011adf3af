// pool.cu -- serving pool (continuous batching) entry points.
#include "fastsv_internal.h"

namespace fsv {
struct Pool {};
void pool_release(fastsv_ctx* h) {
    delete h->pool;
    h->pool = nullptr;
}
}  // namespace fsv

extern "C" {
fastsv_status fastsv_pool_create(fastsv_t, size_t, int32_t) { return FASTSV_ERR_UNSUPPORTED; }
size_t fastsv_pool_bytes(int64_t n, int64_t m) { return (size_t)(n + 1) * 4 + (size_t)m * 4 + (size_t)n * 12; }
fastsv_status fastsv_pool_add(fastsv_t, int64_t, const int32_t*, const int32_t*, int32_t*, int32_t*) {
    return FASTSV_ERR_UNSUPPORTED;
}
fastsv_status fastsv_pool_step(fastsv_t, int32_t, void*) { return FASTSV_ERR_UNSUPPORTED; }
fastsv_status fastsv_pool_poll(fastsv_t, int32_t*, int32_t*, int32_t, int32_t*, int32_t*) {
    return FASTSV_ERR_UNSUPPORTED;
}
fastsv_status fastsv_pool_usage(fastsv_t, int32_t*, size_t*) { return FASTSV_ERR_UNSUPPORTED; }
}

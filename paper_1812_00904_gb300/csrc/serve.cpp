// Serving runtime (continuous batching) -- filled in by the serving milestone.
#include "plan_impl.h"

extern "C" {
spmv_status serve_create(serve_t *out, uint64_t, int32_t, int32_t) {
    if (out) *out = nullptr;
    return gbk::set_error(SPMV_ERR_UNSUPPORTED, "serving not built yet");
}
spmv_status serve_register(serve_t, spmv_plan_t, int32_t *) { return SPMV_ERR_UNSUPPORTED; }
spmv_status serve_register_host(serve_t, int64_t, int64_t, int64_t, int32_t, const int32_t *, const int32_t *,
                                const void *, int32_t, int32_t, int32_t *) {
    return SPMV_ERR_UNSUPPORTED;
}
spmv_status serve_submit(serve_t, int32_t, int32_t, int32_t, const void *, void *, uint64_t *) {
    return SPMV_ERR_UNSUPPORTED;
}
spmv_status serve_poll(serve_t, uint64_t, int32_t *, double *) { return SPMV_ERR_UNSUPPORTED; }
spmv_status serve_wait(serve_t, uint64_t, int32_t) { return SPMV_ERR_UNSUPPORTED; }
spmv_status serve_stats(serve_t, serve_stats_t *) { return SPMV_ERR_UNSUPPORTED; }
spmv_status serve_destroy(serve_t) { return SPMV_OK; }
}

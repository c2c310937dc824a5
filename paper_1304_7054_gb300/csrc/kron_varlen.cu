// Mixed-size batches (placeholder until implemented).
#include "kron_internal.h"

extern "C" {
KRON_API kron_status kron_varlen_plan_create(kron_varlen_plan** plan, int, const kron_class_desc*, int64_t,
                                             const int32_t*, const int64_t*, const int64_t*, kron_dtype,
                                             kron_compute) {
    if (plan) *plan = nullptr;
    return KRON_ERR_NOT_SUPPORTED;
}
KRON_API kron_status kron_varlen_workspace_size(const kron_varlen_plan*, size_t*) { return KRON_ERR_NOT_SUPPORTED; }
KRON_API kron_status kron_varlen_execute(kron_varlen_plan*, const void*, void*, void*, size_t, kron_stream_t) {
    return KRON_ERR_NOT_SUPPORTED;
}
KRON_API kron_status kron_varlen_tune(kron_varlen_plan*, const void*, void*, void*, size_t, kron_stream_t) {
    return KRON_ERR_NOT_SUPPORTED;
}
KRON_API kron_status kron_varlen_plan_destroy(kron_varlen_plan*) { return KRON_OK; }
}

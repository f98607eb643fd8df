// pending.cu -- entry points whose kernels are not written yet.
#include "api_common.h"

using namespace dmrg;

extern "C" {

dmrg_status dmrg_autotune_rotate_ops(dmrg_handle h, const double*, int64_t, int, int64_t,
                                     const void*, int, int64_t, void*, dmrg_precision, void*,
                                     size_t, dmrg_stream_t) {
    return fail(h, DMRG_ERR_UNSUPPORTED, "autotuner not built yet");
}

dmrg_status dmrg_rotate_ops_backward_workspace(dmrg_handle h, int64_t, int64_t, int, int64_t,
                                               dmrg_precision, size_t*) {
    return fail(h, DMRG_ERR_UNSUPPORTED, "backward not built yet");
}

dmrg_status dmrg_rotate_ops_backward(dmrg_handle h, const double*, int64_t, int, int64_t,
                                     const void*, const void*, int, int64_t, void*, double*,
                                     dmrg_precision, void*, size_t, dmrg_stream_t) {
    return fail(h, DMRG_ERR_UNSUPPORTED, "backward not built yet");
}

dmrg_status dmrg_blocked_plan_create(dmrg_handle h, const dmrg_qn_sector*, int32_t,
                                     const dmrg_qn_shift*, int32_t, const dmrg_qn_sector*, int32_t,
                                     const dmrg_qn_shift*, int64_t, dmrg_blocked_plan*) {
    return fail(h, DMRG_ERR_UNSUPPORTED, "blocked path not built yet");
}
dmrg_status dmrg_blocked_plan_destroy(dmrg_blocked_plan) { return DMRG_ERR_UNSUPPORTED; }
dmrg_status dmrg_blocked_plan_sizes(dmrg_blocked_plan, dmrg_precision, int64_t*, int64_t*,
                                    int64_t*, size_t*) {
    return DMRG_ERR_UNSUPPORTED;
}
dmrg_status dmrg_blocked_plan_stats(dmrg_blocked_plan, int64_t*, int64_t*, double*) {
    return DMRG_ERR_UNSUPPORTED;
}
dmrg_status dmrg_rotate_ops_blocked(dmrg_handle h, dmrg_blocked_plan, const double*, const void*,
                                    int, void*, dmrg_precision, void*, size_t, dmrg_stream_t) {
    return fail(h, DMRG_ERR_UNSUPPORTED, "blocked path not built yet");
}

}  // extern "C"

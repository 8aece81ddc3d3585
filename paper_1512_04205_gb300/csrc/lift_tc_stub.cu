#include "cdmd_internal.cuh"
namespace cdmd {
cdmd_status launch_lift_tc(cdmd_ctx*, const uint8_t*, int64_t, int, int64_t, const double*, int, const int32_t*, int, float*, cudaStream_t) {
    return fail(CDMD_ERR_UNSUPPORTED, "BF16X2 lift not built yet");
}
}

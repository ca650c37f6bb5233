// Trailing update of the blocked Householder QR on the 5th-generation tensor
// cores (tcgen05, TMEM accumulators), split TF32x3 precision.  Placeholder until
// the tensor-core kernel lands: reports that the path is unavailable so the
// SIMT update is used.
#include "common.cuh"
#include "qr.cuh"

int fl_trailing_tc_f32(fastlsq_ctx *ctx, float *, int64_t, int64_t, int64_t, int, int, int64_t,
                       const float *)
{
    return fl_fail(ctx, FASTLSQ_ERR_INVALID, "tensor-core trailing update not built");
}

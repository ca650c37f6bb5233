// Self-test of the bounded device waits (failure detection; no counterpart in the
// paper).  Each kernel waits on something that never happens, with a spin budget the
// caller gives, exactly as the library's real waits do: the mbarrier wait of the
// tensor-core kernels (tc::mbar_wait) on a barrier nobody arrives on, and the grid
// barrier of the cooperative kernels (grid_sync) that one CTA never reaches.  When the
// budget runs out the kernel raises FL_DEVERR_TIMEOUT in the context's device flag and
// returns; fastlsq_sync then reports FASTLSQ_ERR_TIMEOUT and resets the flag and the
// barrier state, and the context stays usable.
#include "common.cuh"
#include "gridsync.cuh"
#include "tc_common.cuh"

namespace {

__global__ void k_wait_mbarrier(long long budget, int *flag)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);                 // one arrival expected; none comes
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (!tc::mbar_wait(&bar, 0u, budget)) atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
    }
}

// two CTAs (cooperative launch): CTA 1 leaves without arriving, CTA 0 waits
__global__ void k_wait_grid(GridBar *gbar, long long budget, int *flag)
{
    __shared__ volatile int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    if (blockIdx.x == 1) return;
    grid_sync(gbar, gridDim.x, flag, &s_abort, budget);
}

}  // namespace

extern "C" int fastlsq_selftest_wait(fastlsq_ctx *ctx, int32_t which, int64_t budget_cycles)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (budget_cycles < 0 || budget_cycles > 4000000000ll || (which != 0 && which != 1))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "selftest_wait: which 0 or 1, budget 0..4e9 cycles");
    cudaError_t e;
    if (which == 0) {
        k_wait_mbarrier<<<1, 32, 0, ctx->stream>>>((long long)budget_cycles, ctx->d_flag);
        e = cudaGetLastError();
    } else {
        GridBar *gbar = (GridBar *)ctx->d_grid_bar;
        long long budget = budget_cycles;
        int *flag = ctx->d_flag;
        void *args[] = {(void *)&gbar, (void *)&budget, (void *)&flag};
        e = cudaLaunchCooperativeKernel((const void *)k_wait_grid, dim3(2), dim3(32), args, 0, ctx->stream);
    }
    return e == cudaSuccess ? 0 : fl_cuda(ctx, e, "selftest_wait launch");
}

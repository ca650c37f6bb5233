// Grid-wide barrier for cooperative launches (every CTA resident).  Thread 0 of
// each CTA arrives on a counter and spins on a generation word for at most about
// a second of SM clocks; on timeout it raises the device error flag and the CTA
// leaves the kernel (the host reports FASTLSQ_ERR_TIMEOUT and resets the barrier).
#pragma once
#include "common.cuh"

struct GridBar {
    unsigned count;
    unsigned gen;
};

// give up after about a second of spinning (2e9 SM clocks)
constexpr long long BAR_SPIN_CLOCKS = 2000000000ll;

__device__ __forceinline__ bool grid_sync(GridBar *bar, unsigned nblocks, int *flag,
                                          volatile int *s_abort, long long spin_clocks = BAR_SPIN_CLOCKS)
{
    __syncthreads();
    if (threadIdx.x == 0 && !*s_abort) {
        volatile unsigned *vgen = &bar->gen;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                if (clock64() - t0 > spin_clocks) {
                    atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
                    *s_abort = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *s_abort == 0;
}

// Completion of the Y = V^T C partial sums of a trailing update, as a two-level tree
// so that no CTA adds more than a few dozen partials after the others finish: the
// last CTA of each group of TREE_GS splits of a column tile (counted with an atomic
// per group) adds the group's partials in split order and stores the sum in the
// group's first slot; the last group to finish (an atomic per tile) adds the group
// sums in group order, so the result does not depend on which CTAs finish last, and
// forms Z = T^T Y (T upper triangular) for the tile -- or, with TFWD, Z = T Y (the
// reflectors applied as Q = H_0 ... H_{P-1}, H_p = I - V T V^T, instead of Q^T).  The counters are reset for the
// next panel.  Z is stored [l][c] with row stride nct, or (Zimg) as the tensor-core
// operand image of the tile: Z^T split into tf32 hi and lo parts, each 128 rows (c)
// of 128 bytes (l) in the K-major 128-byte-swizzled layout.
#pragma once
#include "common.cuh"
#include "tc_common.cuh"

constexpr int TREE_GS = 16;        // splits per group
constexpr int TREE_MAXG = 32;      // groups per column tile (splits <= 512)
// counters of column tile t: [t * TREE_STRIDE] the tile's, the next TREE_MAXG its groups'
constexpr int TREE_STRIDE = 1 + TREE_MAXG;
constexpr int TREE_MAX_SPLITS = TREE_GS * TREE_MAXG;

template <typename T, int NB, int COLS, int THREADS, bool IMG = false, bool TFWD = false>
__device__ __forceinline__ void trail_finish_z(T *__restrict__ Ypart, int nsplit, int64_t nct,
                                               int64_t cbase, const T *__restrict__ Tblk,
                                               T *__restrict__ Z, int *counter, int *gcounter, T *scratch)
{
    static_assert(!IMG || (NB == 32 && COLS == 128), "image tiles: 128 columns x 32 l");
    static_assert((NB * COLS) % THREADS == 0, "tile");
    constexpr int ITEMS = NB * COLS / THREADS;
    __shared__ int s_last;
    const int g = (int)blockIdx.y / TREE_GS;
    const int ngroups = (nsplit + TREE_GS - 1) / TREE_GS;
    const int gsz = min(TREE_GS, nsplit - g * TREE_GS);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(gcounter + g, 1) == gsz - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    T *sY = scratch;                    // [NB][COLS]
    T *sT = scratch + NB * COLS;        // [NB * NB], T(q, l) at q + l * NB
    T acc[ITEMS];
    // adds partials first, first + step, ... (count of them) in that order, 8 at a time
    // so that 8 x ITEMS independent loads are in flight per round
    auto sum_slots = [&](int first, int count, int step) {
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) acc[it] = T(0);
        int q0 = 0;
        for (; q0 + 8 <= count; q0 += 8) {
#pragma unroll
            for (int it = 0; it < ITEMS; ++it) {
                const int idx = it * THREADS + threadIdx.x;
                const int l = idx / COLS, cc = idx % COLS;
                const int64_t c = cbase + cc;
                if (c < nct) {
                    const T *src = Ypart + ((int64_t)(first + q0 * step) * NB + l) * nct + c;
                    const int64_t st = (int64_t)step * NB * nct;
                    T a[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) a[q] = __ldcg(src + q * st);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[it] += a[q];
                }
            }
        }
        for (; q0 < count; ++q0) {
#pragma unroll
            for (int it = 0; it < ITEMS; ++it) {
                const int idx = it * THREADS + threadIdx.x;
                const int l = idx / COLS, cc = idx % COLS;
                const int64_t c = cbase + cc;
                if (c < nct) acc[it] += __ldcg(Ypart + ((int64_t)(first + q0 * step) * NB + l) * nct + c);
            }
        }
    };
    sum_slots(g * TREE_GS, gsz, 1);
    if (threadIdx.x == 0) gcounter[g] = 0;
    if (ngroups > 1) {
        // the group's sum goes to its first slot (its partials are all read by now)
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const int idx = it * THREADS + threadIdx.x;
            const int l = idx / COLS, cc = idx % COLS;
            const int64_t c = cbase + cc;
            if (c < nct) __stcg(Ypart + ((int64_t)(g * TREE_GS) * NB + l) * nct + c, acc[it]);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1) == ngroups - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        sum_slots(0, ngroups, TREE_GS);
    }
    for (int idx = threadIdx.x; idx < NB * NB; idx += THREADS) sT[idx] = Tblk[idx];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) sY[it * THREADS + threadIdx.x] = acc[it];
    __syncthreads();
    // Z(l, c) = sum_{q <= l} T(q, l) Y(q, c) (TFWD: sum_{q >= l} T(l, q) Y(q, c)): the
    // thread keeps its column c of Y in registers
    // and forms its ITEMS rows l = h + R it at once (R = THREADS / COLS, h = tid / COLS, the
    // same for a whole warp, so T's entries are broadcast reads)
    static_assert(THREADS % COLS == 0, "threads cover whole columns");
    constexpr int R = THREADS / COLS;
    const int cc = threadIdx.x % COLS, h = threadIdx.x / COLS;
    const int64_t c = cbase + cc;
    T y[NB], z[ITEMS];
#pragma unroll
    for (int q = 0; q < NB; ++q) y[q] = sY[q * COLS + cc];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) z[it] = T(0);
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const int l = h + R * it;
            if constexpr (TFWD) {
                if (q >= l) z[it] += sT[l + q * NB] * y[q];
            } else {
                if (q <= l) z[it] += sT[q + l * NB] * y[q];
            }
        }
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
        const int l = h + R * it;
        if constexpr (IMG) {
            float hi, lo;
            tc::split_tf32((float)(c < nct ? z[it] : T(0)), hi, lo);
            float *img = reinterpret_cast<float *>(Z) + (cbase / COLS) * (2 * COLS * 32);
            const uint32_t off = tc::sw128_offset((uint32_t)cc, (uint32_t)l) >> 2;
            img[off] = hi;
            img[COLS * 32 + off] = lo;
        } else {
            if (c < nct) Z[(int64_t)l * nct + c] = z[it];
        }
    }
    if (threadIdx.x == 0) *counter = 0;
}

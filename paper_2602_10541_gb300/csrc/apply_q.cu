// y <- Q^T y (transpose) or Q y with the compact-WY factors of the blocked QR
// (panel width 32), on one cluster of up to 16 CTAs, one thread per row.
//
// Per panel p (order p = 0.. for Q^T, reversed for Q):
//   s_l = sum_i V(i, l) y_i            (row-parallel, warp reduce-scatter, CTA sum)
//   exchange of the 32 CTA partials between the ranks (asynchronous DSMEM stores
//   that count down the receiver's barrier; no cluster-wide barrier)
//   w = T^T s (Q^T) or w = T s (Q)     (every warp, same order: identical on all ranks)
//   y_i -= sum_l V(i, l) w_l
// The 32 entries V(i, 0..31) of the next panel are loaded into registers while the
// current panel is applied.  Waits are bounded (about a second of SM clock); on
// timeout the device flag is raised and the kernel returns at the next panel.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "qr.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int AQC_NB = 32;
constexpr int AQC_CS_MAX = 16;
constexpr int AQC_MAX_THREADS = 640;
constexpr long long AQC_WAIT = 2000000000ll;

__device__ __forceinline__ uint32_t aq_map_rank(const void *p, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(tc::smem_addr(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void aq_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void aq_bulk_to_rank(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(dst), "r"(tc::smem_addr(src)), "r"(bytes), "r"(bar) : "memory");
}

// V(i, l) of the panel starting at column k, for all 32 l (zero above the panel,
// unit diagonal, zero for columns past the factor)
template <typename T>
__device__ __forceinline__ void aq_load_v(const T *__restrict__ F, int64_t ld, int64_t n, int64_t k,
                                          int64_t i, bool row_ok, T (&v)[AQC_NB])
{
#pragma unroll
    for (int l = 0; l < AQC_NB; ++l) {
        const int64_t col = k + l;
        T x = T(0);
        if (row_ok && col < n && i >= col) x = (i == col) ? T(1) : F[i + col * ld];
        v[l] = x;
    }
}

// lane l returns sum over the warp of vals[l]  (31 shuffles)
template <typename T>
__device__ __forceinline__ T aq_reduce_scatter(T (&vals)[AQC_NB], int lane)
{
#pragma unroll
    for (int s = AQC_NB / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int q = 0; q < s; ++q) {
            const T send = up ? vals[q] : vals[q + s];
            const T keep = up ? vals[q + s] : vals[q];
            vals[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return vals[0];
}

template <typename T>
__global__ void __launch_bounds__(AQC_MAX_THREADS, 1)
k_apply_q_cluster(const T *__restrict__ F, int64_t ld, int64_t m_aug, int64_t n,
                  const T *__restrict__ Tall, T *__restrict__ y, int transpose, int *flag)
{
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ T red[2][AQC_MAX_THREADS / 32][AQC_NB + 1];   // by step parity: a warp may
                                                              // still read step s while another
                                                              // writes step s + 1
    __shared__ __align__(16) T xbuf[2][AQC_CS_MAX][AQC_NB + 4];   // 16-byte rows for bulk copies
    __shared__ __align__(16) T part[2][AQC_NB];
    __shared__ T sT[2][AQC_NB][AQC_NB + 1];                    // the panel's T block, by parity
    __shared__ uint64_t xbar[2];
    __shared__ volatile int s_abort;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int64_t i = (int64_t)rank * blockDim.x + threadIdx.x;
    const bool row_ok = i < m_aug;
    T yi = row_ok ? y[i] : T(0);
    const int npan = (int)((n + AQC_NB - 1) / AQC_NB);
    if (threadIdx.x == 0) {
        tc::mbar_init(&xbar[0], 1);
        tc::mbar_init(&xbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    cluster.sync();
    const uint32_t xbytes = (uint32_t)CS * AQC_NB * (uint32_t)sizeof(T);
    T vn[AQC_NB];
    if (npan > 0) aq_load_v(F, ld, n, (int64_t)(transpose ? 0 : npan - 1) * AQC_NB, i, row_ok, vn);
    // the T block of the next panel, prefetched like V (entries tid + h blockDim, blockDim >= 128)
    T tn[8];
    auto load_t = [&](int pp) {
        const T *Tb = Tall + (int64_t)pp * AQC_NB * AQC_NB;        // T(q, l) at q + 32 l
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int idx = threadIdx.x + h * blockDim.x;
            tn[h] = (idx < AQC_NB * AQC_NB) ? Tb[idx] : T(0);
        }
    };
    if (npan > 0) load_t(transpose ? 0 : npan - 1);
    for (int step = 0; step < npan; ++step) {
        const int p = transpose ? step : npan - 1 - step;
        const int par = step & 1;
        T v[AQC_NB];
#pragma unroll
        for (int l = 0; l < AQC_NB; ++l) v[l] = vn[l];
        if (step + 1 < npan) {
            const int pn = transpose ? step + 1 : npan - 2 - step;
            aq_load_v(F, ld, n, (int64_t)pn * AQC_NB, i, row_ok, vn);
        }
        if (threadIdx.x == 0) aq_expect_tx(&xbar[par], xbytes);
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int idx = threadIdx.x + h * blockDim.x;
            if (idx < AQC_NB * AQC_NB) sT[par][idx % AQC_NB][idx / AQC_NB] = tn[h];
        }
        if (step + 1 < npan) load_t(transpose ? step + 1 : npan - 2 - step);
        // s_l: warp partials, then the CTA's partial sent to every rank
        T prod[AQC_NB];
#pragma unroll
        for (int l = 0; l < AQC_NB; ++l) prod[l] = v[l] * yi;
        red[par][warp][lane] = aq_reduce_scatter(prod, lane);
        __syncthreads();
        if (s_abort) break;                              // uniform after the barrier
        if (warp == 0) {
            // the CTA's 32 partials go to every rank as one bulk copy each
            T s = T(0);
            for (int w = 0; w < nwarps; ++w) s += red[par][w][lane];
            part[par][lane] = s;
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane < CS)
                aq_bulk_to_rank(aq_map_rank(&xbuf[par][rank][0], lane), part[par], AQC_NB * sizeof(T),
                                aq_map_rank(&xbar[par], lane));
        }
        if (!tc::mbar_wait(&xbar[par], (uint32_t)(step >> 1) & 1u, AQC_WAIT)) {
            s_abort = 1;
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        }
        T sl = T(0);
        for (int q = 0; q < CS; ++q) sl += xbuf[par][q][lane];
        // w = T^T s (Q^T) or T s (Q), T from shared memory
        T wl = T(0);
#pragma unroll
        for (int q = 0; q < AQC_NB; ++q) {
            const T sq = __shfl_sync(FULL, sl, q);
            if (transpose) { if (q <= lane) wl += sT[par][q][lane] * sq; }
            else { if (q >= lane) wl += sT[par][lane][q] * sq; }
        }
        T upd = T(0);
#pragma unroll
        for (int l = 0; l < AQC_NB; ++l) upd += v[l] * __shfl_sync(FULL, wl, l);
        yi -= upd;
    }
    if (row_ok) y[i] = yi;
    cluster.sync();    // no CTA leaves while another may still store into its shared memory
}

}  // namespace

// 1 when the cluster kernel cannot take the shape (the caller uses the grid kernel)
template <typename T>
int fl_apply_q_cluster(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t m_aug, int64_t n, int nb,
                       const T *Tall, T *y, int transpose)
{
    if (nb != AQC_NB) return 1;
    int CS = AQC_CS_MAX;
    while (CS > 1 && fl_cdiv(m_aug, CS) < 128) CS >>= 1;
    const int64_t threads = std::max<int64_t>(128, fl_round_up(fl_cdiv(m_aug, CS), 32));   // >= 128: T prefetch
    if (threads > AQC_MAX_THREADS) return 1;
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_apply_q_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "cudaFuncSetAttribute");
        attr_once.done(ctx->device);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FL_PROF(ctx, FASTLSQ_K_APPLY_Q);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_apply_q_cluster<T>, F, ld, m_aug, n, Tall, y, transpose,
                                       ctx->d_flag);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "cluster apply_q launch");
    return 0;
}
template int fl_apply_q_cluster<float>(fastlsq_ctx *, const float *, int64_t, int64_t, int64_t, int,
                                       const float *, float *, int);

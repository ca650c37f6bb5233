// Register-resident panel factorisation for the FP32 factor (panel width 32),
// on a cluster of up to 16 CTAs of 1024 threads.
//
// Lane l of every warp holds column l of the panel; warp w holds RW consecutive
// rows of its CTA's slice in registers, so a column step touches no shared memory
// in its update pass: a_rj comes from a shuffle, the updated a_r,j+1 (for the next
// column's dot products) from a second shuffle.  Per column j:
//   1. the CTA's partial sums (one per lane/column, accumulated by the previous
//      update pass) are reduced across the 32 warps, warp c reducing column c;
//   2. each CTA stores its 32 partials, plus rank 0 the diagonal row a_j., into
//      every rank's shared memory (DSMEM) and the cluster synchronises once;
//   3. warp c sums the CL partials of column c in a fixed order (every rank gets
//      bit-identical sums); warp j forms the reflector of column j;
//   4. every lane updates its rows with H_j and accumulates the next column's
//      dot products (l > j) and the Gram entries v_l^T v_j (l < j) for T.
// Reflector convention, Gram/T recurrence and output layout are those of the
// shared-memory panel kernel in qr.cu (LAPACK sign choice, T built at the end).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "qr.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int PR_NB = 32;
constexpr int PR_THREADS = 1024;
constexpr int PR_CL_MAX = 16;
constexpr int PR_XLD = 33;                   // padded stride of the exchange buffer

struct PrLayout {
    // offsets in floats
    static __host__ __device__ size_t red(int rpc) { return (size_t)rpc * 33; }
    static __host__ __device__ size_t xbuf(int rpc) { return red(rpc) + 32 * 33; }
    static __host__ __device__ size_t dsum(int rpc) { return xbuf(rpc) + 2 * (PR_CL_MAX + 1) * PR_XLD; }
    static __host__ __device__ size_t sc(int rpc) { return dsum(rpc) + 32; }
    static __host__ __device__ size_t diag(int rpc) { return sc(rpc) + 32; }
    static __host__ __device__ size_t Tm(int rpc) { return diag(rpc) + 32; }
    static __host__ __device__ size_t G(int rpc) { return Tm(rpc) + 32 * 33; }
    static __host__ __device__ size_t tauv(int rpc) { return G(rpc) + 32 * 33; }
    static __host__ __device__ size_t bytes(int rpc) { return sizeof(float) * (tauv(rpc) + 32); }
};

template <int RW>
__global__ void __launch_bounds__(PR_THREADS, 1)
k_panel_reg(float *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols,
            float *__restrict__ tau_out, float *__restrict__ T_out, int *flag)
{
    constexpr int rpc = 32 * RW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) float psm[];
    float *S = psm;
    float *red = psm + PrLayout::red(rpc);
    float *xbuf = psm + PrLayout::xbuf(rpc);
    float *dsum = psm + PrLayout::dsum(rpc);
    float *sc = psm + PrLayout::sc(rpc);
    float *diag = psm + PrLayout::diag(rpc);
    float *Tm = psm + PrLayout::Tm(rpc);
    float *G = psm + PrLayout::G(rpc);
    float *tauv = psm + PrLayout::tauv(rpc);

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int64_t mp = m - k;
    const int64_t c0 = (int64_t)rank * rpc;
    const int nown = (int)fl_max64(0, fl_min64(rpc, mp - c0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = lane;
    const int64_t g0 = c0 + (int64_t)warp * RW;    // panel-local row of register row 0

    // stage the slice through shared memory (coalesced along the columns of F)
    for (int idx = threadIdx.x; idx < rpc * 32; idx += PR_THREADS) {
        const int c = idx / rpc, r = idx % rpc;
        S[r * 33 + c] = (r < nown && c < ncols) ? F[(k + c0 + r) + (k + c) * ld] : 0.f;
    }
    for (int idx = threadIdx.x; idx < 2 * 32 * 33; idx += PR_THREADS) Tm[idx] = 0.f;   // Tm and G
    __syncthreads();
    float p[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) p[r] = S[(warp * RW + r) * 33 + l];
    if (g0 == 0) diag[l] = p[0];                    // diagonal row 0 (rank 0, warp 0)
    // dot products of column 0 with every column over rows 1..
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const float a0 = __shfl_sync(FULL, p[r], 0);
        if (g0 + r > 0) acc = fmaf(a0, p[r], acc);
    }

    for (int j = 0; j <= ncols; ++j) {
        const int par = j & 1;
        float *xb = xbuf + par * (PR_CL_MAX + 1) * PR_XLD;
        red[warp * 33 + lane] = acc;
        __syncthreads();
        {
            // warp c reduces column c over the 32 warps and sends the CTA's partial
            const int c = warp;
            float s = red[lane * 33 + c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
            s = __shfl_sync(FULL, s, 0);
            if (lane < CL) {
                float *rb = cluster.map_shared_rank(xb, lane);
                rb[rank * PR_XLD + c] = s;
                if (rank == 0) rb[PR_CL_MAX * PR_XLD + c] = (j < ncols) ? diag[c] : 0.f;
            }
        }
        cluster.sync();
        {
            // warp c sums the CL partials of column c (fixed order, same on every rank)
            const int c = warp;
            float v = (lane < CL) ? xb[lane * PR_XLD + c] : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            v = __shfl_sync(FULL, v, 0);
            if (lane == 0) {
                dsum[c] = v;
                if (rank == 0 && j >= 1 && c < j - 1) G[c * 33 + (j - 1)] = v;
                if (c == j && j < ncols) {
                    // reflector of column j: v = 1 at row j, a(j+1:)/(a_jj - beta) below
                    const float ss = v, ajj = xb[PR_CL_MAX * PR_XLD + j];
                    float beta = ajj, tj = 0.f, inv = 0.f;
                    if (!isfinite(ss) || !isfinite(ajj)) {
                        atomicCAS(flag, 0, FL_DEVERR_NONFINITE);
                    } else if (ss > 0.f) {
                        const float nrm = sqrtf(ajj * ajj + ss);
                        beta = (ajj >= 0.f) ? -nrm : nrm;
                        tj = (beta - ajj) / beta;
                        inv = 1.f / (ajj - beta);
                    }
                    sc[0] = beta;
                    sc[1] = tj;
                    sc[2] = inv;
                    if (rank == 0) tauv[j] = tj;
                }
            }
        }
        if (j == ncols) break;
        __syncthreads();
        const float beta = sc[0], tj = sc[1], inv = sc[2];
        const float wl = (l > j) ? tj * (xb[PR_CL_MAX * PR_XLD + l] + inv * dsum[l]) : 0.f;
        const int jn = (j + 1) & 31;
        acc = 0.f;
        if (g0 >= j + 2) {
            // every row of this warp lies below the next diagonal row
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const float vj = __shfl_sync(FULL, p[r], j) * inv;
                const float nl = fmaf(-wl, vj, p[r]);
                const float nx = __shfl_sync(FULL, nl, jn);
                p[r] = (l == j) ? vj : nl;
                const float f = (l > j) ? nx : ((l < j) ? vj : 0.f);
                acc = fmaf(f, nl, acc);
            }
        } else {
            // rows at or above j + 1 (rank 0's first warps): row j takes beta, row j + 1
            // is the next diagonal row and stays out of the next column's dot products
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const int64_t g = g0 + r;                   // uniform across the warp
                const float pj = __shfl_sync(FULL, p[r], j);
                const float vj = (g == j) ? 1.f : pj * inv;
                const float nl = fmaf(-wl, vj, p[r]);
                const float nx = __shfl_sync(FULL, nl, jn);
                if (g < j) continue;
                const float nv = (l == j) ? ((g == j) ? beta : vj) : nl;
                p[r] = nv;
                const float f = (l < j) ? vj : ((l > j && g > j + 1) ? nx : 0.f);
                acc = fmaf(f, nl, acc);
                if (g == j + 1) diag[l] = nv;
            }
        }
    }

    // write the slice back (coalesced through shared memory); rank 0 forms T
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RW; ++r) S[(warp * RW + r) * 33 + l] = p[r];
    __syncthreads();
    for (int idx = threadIdx.x; idx < rpc * 32; idx += PR_THREADS) {
        const int c = idx / rpc, r = idx % rpc;
        if (r < nown && c < ncols) F[(k + c0 + r) + (k + c) * ld] = S[r * 33 + c];
    }
    if (rank == 0 && warp == 0) {
        // T(c, c) = tau_c ; T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c)   (lane = row)
        for (int c = 0; c < ncols; ++c) {
            const float tc = tauv[c];
            float sum = 0.f;
            if (lane < c)
                for (int q = lane; q < c; ++q) sum += Tm[lane * 33 + q] * G[q * 33 + c];
            __syncwarp();
            if (lane < c) Tm[lane * 33 + c] = -tc * sum;
            if (lane == c) Tm[c * 33 + c] = tc;
            __syncwarp();
        }
        tau_out[lane] = (lane < ncols) ? tauv[lane] : 0.f;
        for (int idx = lane; idx < PR_NB * PR_NB; idx += 32) {
            const int col = idx / PR_NB, row = idx % PR_NB;
            T_out[idx] = (col < ncols && row < ncols) ? Tm[row * 33 + col] : 0.f;
        }
    }
    // no CTA leaves while another may still store into its shared memory
    cluster.sync();
}

template <int RW>
int launch_panel_reg(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                     int CL, float *tau, float *Tblk)
{
    const size_t smem = PrLayout::bytes(32 * RW);
    static bool attr_done = false;   // per process; attributes are per function
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_panel_reg<RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_panel_reg<RW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "cudaFuncSetAttribute");
        attr_done = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(PR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FL_PROF(ctx, FASTLSQ_K_PANEL);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_panel_reg<RW>, F, ld, k, m_aug, ncols, tau, Tblk, ctx->d_flag);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "register panel launch");
    return 0;
}

}  // namespace

int fl_panel_reg_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                     float *tau, float *Tblk)
{
    const int64_t mp = m_aug - k;
    // enough CTAs that each warp holds at most 24 rows, no more than needed for 8
    const int CL = (int)std::min<int64_t>(PR_CL_MAX, std::max<int64_t>(1, fl_cdiv(mp, 32 * 8)));
    const int64_t rpw = fl_cdiv(fl_cdiv(mp, CL), 32);
    if (rpw <= 8) return launch_panel_reg<8>(ctx, F, ld, k, m_aug, ncols, CL, tau, Tblk);
    if (rpw <= 12) return launch_panel_reg<12>(ctx, F, ld, k, m_aug, ncols, CL, tau, Tblk);
    if (rpw <= 16) return launch_panel_reg<16>(ctx, F, ld, k, m_aug, ncols, CL, tau, Tblk);
    if (rpw <= 20) return launch_panel_reg<20>(ctx, F, ld, k, m_aug, ncols, CL, tau, Tblk);
    if (rpw <= 24) return launch_panel_reg<24>(ctx, F, ld, k, m_aug, ncols, CL, tau, Tblk);
    return 1;   // too tall for registers: the caller uses the shared-memory panel
}

bool fl_panel_reg_fits(int64_t mp)
{
    const int64_t CL = std::min<int64_t>(PR_CL_MAX, std::max<int64_t>(1, fl_cdiv(mp, 32 * 8)));
    return fl_cdiv(fl_cdiv(mp, CL), 32) <= 24;
}

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
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int PR_NB = 32;
constexpr int PR_THREADS = 1024;
constexpr int PR_CL_MAX = 16;
constexpr int PR_XLD = 36;                   // row stride of the exchange buffer (16-byte rows)
constexpr int PR_STAGE_U = 8;                // loads in flight per thread when staging
constexpr long long PR_SPIN = 2000000000ll;  // SM cycles (about a second) before an exchange wait gives up

// shared::cluster address of the same shared-memory object in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(const void *p, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(tc::smem_addr(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

// store 16 bytes to another CTA's shared memory and count them down on its barrier
__device__ __forceinline__ void st_async_v4(uint32_t addr, float4 v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];\n"
                 :: "r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar) : "memory");
}

// bulk copy of `bytes` (multiple of 16) from this CTA's shared memory into another
// CTA's, counted down on the receiver's barrier
__device__ __forceinline__ void bulk_to_rank(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(dst), "r"(tc::smem_addr(src)), "r"(bytes), "r"(bar) : "memory");
}

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
    // with the previous panel's update fused in front: its V slice and the Y/Z buffers
    static __host__ __device__ size_t sv(int rpc) { return tauv(rpc) + 32; }        // [rpc][36]
    static __host__ __device__ size_t yp(int rpc) { return sv(rpc) + (size_t)rpc * 36; }  // [32][32]
    static __host__ __device__ size_t rs(int rpc) { return yp(rpc) + 1024; }        // [48][32]
    static __host__ __device__ size_t ys(int rpc) { return rs(rpc) + 48 * 32; }     // [32][32]
    static __host__ __device__ size_t yf(int rpc) { return ys(rpc) + 1024; }        // [32][32]
    static __host__ __device__ size_t zs(int rpc) { return yf(rpc) + 1024; }        // [32][33]
    static __host__ __device__ size_t tp(int rpc) { return zs(rpc) + 32 * 33; }     // [32 * 32]
    static __host__ __device__ size_t bytes_fused(int rpc) { return sizeof(float) * (tp(rpc) + 1024); }
};

// The previous panel's update of this panel's columns, fused in front of the panel:
// C -= V (T^T (V^T C)) over rows kp.. with V, T of the panel starting at column kp.
// C sits in registers (lane = column, p[r]) and in S; V in SV; rank 0 also holds the 32
// rows kp..kp+31 of C (CT, in Tm) and the unit lower triangle of V (VT, in G).
//  1. Y partial (32 x 32) of this CTA: thread = (4 x 4 block of Y, one of 16 row groups),
//     sum over the row groups with shuffles;
//  2. reduce-scatter: row l of the partial goes to rank l % CL (128-byte bulk copies),
//     which adds the CL partials in rank order;
//  3. all-gather of the summed rows to every rank (bulk copies): all ranks hold the same Y;
//  4. Z = T^T Y; p[r] -= V(row, :) Z on the register rows; rank 0 writes CT - VT Z back.
template <int RW>
__device__ __forceinline__ void prev_panel_z(int rank, int CL, int nown, float *psm, int *flag,
                                             uint64_t *ybar, volatile int *s_abort)
{
    constexpr int rpc = 32 * RW;
    constexpr unsigned FULL = 0xffffffffu;
    const float *S = psm;
    const float *SV = psm + PrLayout::sv(rpc);
    float *Yp = psm + PrLayout::yp(rpc);
    float *RS = psm + PrLayout::rs(rpc);
    float *YS = psm + PrLayout::ys(rpc);
    float *YF = psm + PrLayout::yf(rpc);
    float *Zs = psm + PrLayout::zs(rpc);
    const float *Tp = psm + PrLayout::tp(rpc);
    float *Tm = psm + PrLayout::Tm(rpc);
    const float *G = psm + PrLayout::G(rpc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // 1. this CTA's partial of Y = V^T C
    {
        const int rg = threadIdx.x & 15, blk = threadIdx.x >> 4, lb = blk >> 3, cb = blk & 7;
        float y[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) y[a][b] = 0.f;
        if (rank == 0)          // the 32 rows above the slice: rows rg and rg + 16 of VT, CT
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = rg + 16 * h;
                float va[4], cc[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) va[a] = G[i * 33 + 4 * lb + a];
#pragma unroll
                for (int b = 0; b < 4; ++b) cc[b] = Tm[i * 33 + 4 * cb + b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) y[a][b] = fmaf(va[a], cc[b], y[a][b]);
            }
#pragma unroll 4
        for (int r = rg; r < nown; r += 16) {
            const float4 v = *reinterpret_cast<const float4 *>(SV + r * 36 + 4 * lb);
            const float va[4] = {v.x, v.y, v.z, v.w};
            float cc[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) cc[b] = S[r * 33 + 4 * cb + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) y[a][b] = fmaf(va[a], cc[b], y[a][b]);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) y[a][b] += __shfl_xor_sync(FULL, y[a][b], o);
        if (rg == 0) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) Yp[(4 * lb + a) * 32 + 4 * cb + b] = y[a][b];
            tc::fence_proxy_async_smem();
        }
    }
    __syncthreads();
    // 2. reduce-scatter
    const int rpo = (32 + CL - 1) / CL;                  // rows per owner, at most
    const int mine = (32 - rank + CL - 1) / CL;          // rows owned by this rank
    if (threadIdx.x == 0) arrive_expect_tx(&ybar[0], (uint32_t)(mine * CL * 128));
    if (threadIdx.x < 32) {
        const int row = threadIdx.x, q = row % CL;
        bulk_to_rank(map_rank(RS + (rank * rpo + row / CL) * 32, q), Yp + row * 32, 128, map_rank(&ybar[0], q));
    }
    if (!tc::mbar_wait(&ybar[0], 0u, PR_SPIN)) {
        *s_abort = 1;
        atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
    }
    for (int idx = threadIdx.x; idx < mine * 32; idx += PR_THREADS) {
        const int lr = idx / 32, c = idx % 32;
        float sum = 0.f;
        for (int src = 0; src < CL; ++src) sum += RS[(src * rpo + lr) * 32 + c];
        YS[lr * 32 + c] = sum;
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    // 3. all-gather
    if (threadIdx.x == 0) arrive_expect_tx(&ybar[1], 32u * 128u);
    for (int idx = threadIdx.x; idx < mine * CL; idx += PR_THREADS) {
        const int lr = idx / CL, q = idx % CL, row = lr * CL + rank;
        bulk_to_rank(map_rank(YF + row * 32, q), YS + lr * 32, 128, map_rank(&ybar[1], q));
    }
    if (!tc::mbar_wait(&ybar[1], 0u, PR_SPIN)) {
        *s_abort = 1;
        atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
    }
    // 4. Z = T^T Y (T(q, l) at Tp[q + 32 l], upper triangular), then the updates
    {
        float z = 0.f;
        for (int q = 0; q <= warp; ++q) z = fmaf(Tp[q + warp * 32], YF[q * 32 + lane], z);
        Zs[warp * 33 + lane] = z;
    }
    __syncthreads();
}

template <int RW>
__device__ __forceinline__ void prev_panel_apply(int rank, int ncols, float *__restrict__ F, int64_t ld,
                                                 int64_t k, int64_t kp, float *psm, float (&p)[RW])
{
    constexpr int rpc = 32 * RW;
    const float *SV = psm + PrLayout::sv(rpc);
    const float *Zs = psm + PrLayout::zs(rpc);
    const float *Tm = psm + PrLayout::Tm(rpc);
    const float *G = psm + PrLayout::G(rpc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int l0 = 0; l0 < 32; l0 += 8) {
        float zc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) zc[i] = Zs[(l0 + i) * 33 + lane];
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const float *v = SV + (r * 32 + warp) * 36 + l0;
            const float4 va = *reinterpret_cast<const float4 *>(v);
            const float4 vb = *reinterpret_cast<const float4 *>(v + 4);
            float u = va.x * zc[0];
            u = fmaf(va.y, zc[1], u);
            u = fmaf(va.z, zc[2], u);
            u = fmaf(va.w, zc[3], u);
            u = fmaf(vb.x, zc[4], u);
            u = fmaf(vb.y, zc[5], u);
            u = fmaf(vb.z, zc[6], u);
            u = fmaf(vb.w, zc[7], u);
            p[r] -= u;
        }
    }
    if (rank == 0) {
        const int i = warp, c = lane;
        float u = 0.f;
        for (int q = 0; q < 32; ++q) u = fmaf(G[i * 33 + q], Zs[q * 33 + c], u);
        if (c < ncols) F[(kp + i) + (k + c) * ld] = Tm[i * 33 + c] - u;
    }
    __syncthreads();
}

template <int RW>
__global__ void __launch_bounds__(PR_THREADS, 1)
k_panel_reg(float *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols,
            float *__restrict__ tau_out, float *__restrict__ T_out, int *flag,
            int64_t kp, const float *__restrict__ Tprev)
{
    constexpr int rpc = 32 * RW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) float psm[];
    float *S = psm;
    float *red = psm + PrLayout::red(rpc);
    float *xbuf = psm + PrLayout::xbuf(rpc);
    float *diag = psm + PrLayout::diag(rpc);
    float *Tm = psm + PrLayout::Tm(rpc);
    float *G = psm + PrLayout::G(rpc);
    float *tauv = psm + PrLayout::tauv(rpc);
    __shared__ uint64_t xbar[2];
    __shared__ uint64_t ybar[2];                     // the fused update's two exchanges
    __shared__ __align__(16) float part[2][32];      // this CTA's partials, by column parity
    __shared__ __align__(16) float pdiag[2][32];     // rank 0: the diagonal row, by parity
    __shared__ volatile int s_abort;

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int64_t mp = m - k;
    const int64_t c0 = (int64_t)rank * rpc;
    const int nown = (int)fl_max64(0, fl_min64(rpc, mp - c0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = lane;
    // register row r of warp w holds CTA row 32 r + w: the rows next to the diagonal
    // (panel rows <= 32) are register rows 0 and 1 of rank 0, spread over all warps
    const int64_t g0 = c0 + warp;                   // panel-local row of register row 0

    // exchange barriers: per phase one local arrival (with the expected byte count) plus
    // the byte counts of the asynchronous DSMEM stores or bulk copies aimed at them
    if (threadIdx.x == 0) {
        tc::mbar_init(&xbar[0], 1);
        tc::mbar_init(&xbar[1], 1);
        tc::mbar_init(&ybar[0], 1);
        tc::mbar_init(&ybar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    cluster.sync();                                  // barriers ready before any remote signal

    // stage the slice through shared memory (coalesced along the columns of F)
    const bool fused = kp >= 0;
    // (loads in groups of PR_STAGE_U per thread, so that many are in flight at once)
#pragma unroll 1
    for (int base = threadIdx.x; base < rpc * 32; base += PR_THREADS * PR_STAGE_U) {
        float v[PR_STAGE_U];
#pragma unroll
        for (int u = 0; u < PR_STAGE_U; ++u) {
            const int idx = base + u * PR_THREADS, c = idx / rpc, r = idx % rpc;
            v[u] = (idx < rpc * 32 && r < nown && c < ncols) ? F[(k + c0 + r) + (k + c) * ld] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < PR_STAGE_U; ++u) {
            const int idx = base + u * PR_THREADS;
            if (idx < rpc * 32) S[(idx % rpc) * 33 + idx / rpc] = v[u];
        }
    }
    float *SV = psm + PrLayout::sv(rpc);
    if (fused) {
        // the previous panel's reflectors (columns kp..kp+31) on this CTA's rows, which
        // lie below that panel's diagonal block; its T; on rank 0 the 32 rows kp..kp+31
        // of this panel's columns (CT, in Tm) and the unit lower triangle of V (VT, in G)
#pragma unroll 1
        for (int base = threadIdx.x; base < rpc * 32; base += PR_THREADS * PR_STAGE_U) {
            float v[PR_STAGE_U];
#pragma unroll
            for (int u = 0; u < PR_STAGE_U; ++u) {
                const int idx = base + u * PR_THREADS, c = idx / rpc, r = idx % rpc;
                v[u] = (idx < rpc * 32 && r < nown) ? F[(k + c0 + r) + (kp + c) * ld] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < PR_STAGE_U; ++u) {
                const int idx = base + u * PR_THREADS;
                if (idx < rpc * 32) SV[(idx % rpc) * 36 + idx / rpc] = v[u];
            }
        }
        float *Tp = psm + PrLayout::tp(rpc);
        for (int idx = threadIdx.x; idx < 1024; idx += PR_THREADS) Tp[idx] = Tprev[idx];
        if (rank == 0)
            for (int idx = threadIdx.x; idx < 1024; idx += PR_THREADS) {
                const int i = idx % 32, c = idx / 32;
                Tm[i * 33 + c] = (c < ncols) ? F[(kp + i) + (k + c) * ld] : 0.f;
                G[i * 33 + c] = (i > c) ? F[(kp + i) + (kp + c) * ld] : ((i == c) ? 1.f : 0.f);
            }
    }
    __syncthreads();
    if (fused) prev_panel_z<RW>(rank, CL, nown, psm, flag, ybar, &s_abort);
    float p[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) p[r] = S[(r * 32 + warp) * 33 + l];
    if (fused) prev_panel_apply<RW>(rank, ncols, F, ld, k, kp, psm, p);
    for (int idx = threadIdx.x; idx < 2 * 32 * 33; idx += PR_THREADS) Tm[idx] = 0.f;   // Tm and G
    __syncthreads();
    if (g0 == 0) diag[l] = p[0];                    // diagonal row 0 (rank 0, warp 0)
    // dot products of column 0 with every column over rows 1..
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const float a0 = __shfl_sync(FULL, p[r], 0);
        if (g0 + 32 * r > 0) acc = fmaf(a0, p[r], acc);
    }

    const uint32_t xbytes = (uint32_t)(CL + 1) * 32u * (uint32_t)sizeof(float);

    for (int j = 0; j <= ncols; ++j) {
        const int par = j & 1;
        float *xb = xbuf + par * (PR_CL_MAX + 1) * PR_XLD;
        if (threadIdx.x == 0) arrive_expect_tx(&xbar[par], xbytes);
        red[warp * 33 + lane] = acc;
        __syncthreads();
        if (s_abort) break;                          // uniform: read after the barrier
        {
            // warp c reduces column c over the 32 warps into this CTA's partial vector
            const int c = warp;
            float s = red[lane * 33 + c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
            if (lane == 0) {
                part[par][c] = s;
                if (rank == 0) pdiag[par][c] = (j < ncols) ? diag[c] : 0.f;
            }
        }
        __syncthreads();
        if (warp < CL) {
            // warp q sends the 32 partials (lanes 0-7, 16 bytes each) and, on rank 0, the
            // diagonal row (lanes 8-15) to rank q with asynchronous DSMEM stores that
            // count the bytes down on rank q's barrier
            const int q = warp;
            const uint32_t rbar = map_rank(&xbar[par], q);
            if (lane < 8)
                st_async_v4(map_rank(xb + rank * PR_XLD + 4 * lane, q),
                            *reinterpret_cast<const float4 *>(&part[par][4 * lane]), rbar);
            else if (lane < 16 && rank == 0)
                st_async_v4(map_rank(xb + PR_CL_MAX * PR_XLD + 4 * (lane - 8), q),
                            *reinterpret_cast<const float4 *>(&pdiag[par][4 * (lane - 8)]), rbar);
        }
        if (!tc::mbar_wait(&xbar[par], (uint32_t)(j >> 1) & 1u, PR_SPIN)) {
            s_abort = 1;                             // every warp leaves at the next barrier
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        }
        // every warp sums the CL partials of every column in the same order, so all
        // warps of all ranks hold bit-identical sums and reflector scalars
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;    // four chains, fixed order
#pragma unroll
        for (int q = 0; q < PR_CL_MAX; q += 4) {
            if (q < CL) d0 += xb[q * PR_XLD + l];
            if (q + 1 < CL) d1 += xb[(q + 1) * PR_XLD + l];
            if (q + 2 < CL) d2 += xb[(q + 2) * PR_XLD + l];
            if (q + 3 < CL) d3 += xb[(q + 3) * PR_XLD + l];
        }
        const float dl = (d0 + d1) + (d2 + d3);
        if (rank == 0 && warp == 0 && j >= 1 && l < j - 1) G[l * 33 + (j - 1)] = dl;
        if (j == ncols) break;
        const float ss = __shfl_sync(FULL, dl, j);
        const float ajj = xb[PR_CL_MAX * PR_XLD + j];
        float beta = ajj, tj = 0.f, inv = 0.f;
        if (!isfinite(ss) || !isfinite(ajj)) {
            if (lane == 0) atomicCAS(flag, 0, FL_DEVERR_NONFINITE);
        } else if (ss > 0.f) {
            // reflector of column j: v = 1 at row j, a(j+1:)/(a_jj - beta) below
            const float nrm = sqrtf(ajj * ajj + ss);
            beta = (ajj >= 0.f) ? -nrm : nrm;
            tj = __fdividef(beta - ajj, beta);       // |beta| >= |ajj| > 0: in range, 2 ulp
            inv = __fdividef(1.f, ajj - beta);
        }
        if (rank == 0 && warp == 0 && lane == 0) tauv[j] = tj;
        const float wl = (l > j) ? tj * (xb[PR_CL_MAX * PR_XLD + l] + inv * dl) : 0.f;
        const int jn = (j + 1) & 31;
        acc = 0.f;
        // register rows 0 and 1 may be rows at or above j + 1 (rank 0): row j takes beta,
        // row j + 1 is the next diagonal row and stays out of the next column's dot
        // products, rows above j are finished rows of R
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int64_t g = g0 + 32 * r;                 // uniform across the warp
            const float pj = __shfl_sync(FULL, p[r], j);
            const float vj = (g == j) ? 1.f : pj * inv;
            const float nl = fmaf(-wl, vj, p[r]);
            const float nx = __shfl_sync(FULL, nl, jn);
            if (g >= j) {
                const float nv = (l == j) ? ((g == j) ? beta : vj) : nl;
                p[r] = nv;
                const float f = (l < j) ? vj : ((l > j && g > j + 1) ? nx : 0.f);
                acc = fmaf(f, nl, acc);
                if (g == j + 1) diag[l] = nv;
            }
        }
        // register rows 2.. are panel rows >= 64, always below the next diagonal row
#pragma unroll
        for (int r = 2; r < RW; ++r) {
            const float vj = __shfl_sync(FULL, p[r], j) * inv;
            const float nl = fmaf(-wl, vj, p[r]);
            const float nx = __shfl_sync(FULL, nl, jn);
            p[r] = (l == j) ? vj : nl;
            const float f = (l > j) ? nx : ((l < j) ? vj : 0.f);
            acc = fmaf(f, nl, acc);
        }
    }

    // write the slice back (coalesced through shared memory); rank 0 forms T
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RW; ++r) S[(r * 32 + warp) * 33 + l] = p[r];
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
                     int CL, float *tau, float *Tblk, int64_t kp, const float *Tprev)
{
    const size_t plain = PrLayout::bytes(32 * RW), fused = PrLayout::bytes_fused(32 * RW);
    const size_t cap = (size_t)ctx->max_smem_optin - 1024;          // static shared memory aside
    const size_t smem = kp >= 0 ? fused : plain;
    if (smem > cap) return 2;
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_panel_reg<RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)std::min(fused > cap ? plain : fused, cap));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_panel_reg<RW>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "cudaFuncSetAttribute");
        attr_once.done(ctx->device);
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_panel_reg<RW>, F, ld, k, m_aug, ncols, tau, Tblk, ctx->d_flag,
                                       kp, Tprev);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "register panel launch");
    return 0;
}

}  // namespace

int fl_panel_reg_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                     float *tau, float *Tblk, int64_t kp, const float *Tprev)
{
    if (ctx->row_panel) {
        const int rc = fl_panel_row_f32(ctx, F, ld, k, m_aug, ncols, tau, Tblk, kp, Tprev);
        if (rc != 1 && rc != 2) return rc;
    }
    const int64_t mp = m_aug - k;
    // enough CTAs that each warp holds at most 24 rows, no more than needed for 8
    const int CL = (int)std::min<int64_t>(PR_CL_MAX, std::max<int64_t>(1, fl_cdiv(mp, 32 * 8)));
    const int64_t rpw = fl_cdiv(fl_cdiv(mp, CL), 32);
#define FL_PANEL_RW(R) \
    if (rpw <= R) return launch_panel_reg<R>(ctx, F, ld, k, m_aug, ncols, CL, tau, Tblk, kp, Tprev);
    FL_PANEL_RW(8) FL_PANEL_RW(12) FL_PANEL_RW(16) FL_PANEL_RW(18) FL_PANEL_RW(20) FL_PANEL_RW(24)
#undef FL_PANEL_RW
    return 1;   // too tall for registers: the caller uses the shared-memory panel
}

bool fl_panel_reg_fits(int64_t mp)
{
    const int64_t CL = std::min<int64_t>(PR_CL_MAX, std::max<int64_t>(1, fl_cdiv(mp, 32 * 8)));
    return fl_cdiv(fl_cdiv(mp, CL), 32) <= 24;
}

bool fl_panel_reg_fused_fits(fastlsq_ctx *ctx, int64_t mp)
{
    if (ctx->row_panel && fl_panel_row_fits(ctx, mp, true)) return true;
    const int64_t CL = std::min<int64_t>(PR_CL_MAX, std::max<int64_t>(1, fl_cdiv(mp, 32 * 8)));
    const int64_t rpw = fl_cdiv(fl_cdiv(mp, CL), 32);
    const int rw = rpw <= 8 ? 8 : rpw <= 12 ? 12 : rpw <= 16 ? 16 : rpw <= 18 ? 18 : rpw <= 20 ? 20 : 24;
    if (rpw > 24) return false;
    return PrLayout::bytes_fused(32 * rw) <= (size_t)ctx->max_smem_optin - 1024;
}

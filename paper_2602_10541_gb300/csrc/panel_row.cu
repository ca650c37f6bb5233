// Row-resident panel factorisation for the FP32 factor (panel width 32): Householder
// QR of the panel (Sec. 2.3, LAPACK sign convention, compact-WY T) on a cluster of up
// to 16 CTAs, one thread per panel row.
//
// Thread t of CTA c holds row c * rows_per_cta + t of the panel, all 32 columns, in
// registers.  Per column j:
//   1. each thread forms the 32 products a_j a_l of its row (rows below j only), the
//      warp reduce-scatters them (lane l gets the warp's sum for column l) and warp 0
//      adds the warps' sums in a fixed order;
//   2. the CTA's 32 sums and, on rank 0, the pivot row a_j. go to every rank as
//      asynchronous DSMEM stores that count down the receiver's barrier;
//   3. every warp adds the ranks' sums in the same fixed order (all threads of all
//      ranks hold bit-identical reflector scalars) and forms w_l = tau v_j^T a_l;
//   4. each thread updates its own row: no shuffles and no shared memory in the
//      update, the row is in the thread's registers (column j picked by selects, so
//      that the column loop stays a loop).
// The sums for l < j are the Gram entries v_l^T v_j of the reflectors (less the
// pivot row's part), from which T = (I + D striu(V^T V))^{-1} D, D = diag(tau), is
// formed at the end by a triangular inverse (one lane per column of T).
//
// With kp >= 0 the kernel first applies the previous panel (its reflectors in F at
// columns kp.., its T in Tprev) to this panel's columns, rows kp.. (the look-ahead
// update): Y = V^T C by register tiles from shared memory, a reduce-scatter and an
// all-gather of Y over the cluster (bulk DSMEM copies), Z = T^T Y, then C -= V Z on
// the row registers.  Loads and stores of the panel are coalesced along the rows of
// F directly from and to the row registers.  Waits are bounded (about a second of
// SM clock): on timeout the device flag is raised and the kernel returns.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "qr.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int RP_NB = 32;
constexpr int RP_CL_MAX = 16;
constexpr int RP_MAX_ROWS = 768;              // rows per CTA
constexpr int RP_XLD = 36;                    // row stride of the exchange buffer (16-byte rows)
constexpr int RP_GLD = 36;                    // row stride of the Gram matrix (float4 rows)
constexpr long long RP_SPIN = 2000000000ll;   // SM cycles (about a second) before a wait gives up

__device__ __forceinline__ uint32_t rp_map(const void *p, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(tc::smem_addr(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void rp_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void rp_st_async_v4(uint32_t addr, float4 v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];\n"
                 :: "r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar) : "memory");
}

// contiguous global -> own shared memory copy (16-byte aligned, multiple of 16 bytes)
__device__ __forceinline__ void rp_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(tc::smem_addr(dst)), "l"(src), "r"(bytes), "r"(tc::smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void rp_bulk_to_rank(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(dst), "r"(tc::smem_addr(src)), "r"(bytes), "r"(bar) : "memory");
}

// lane l returns the warp's sum of vals[l]  (31 shuffles, vals is overwritten)
__device__ __forceinline__ float rp_reduce_scatter(float (&vals)[RP_NB], int lane)
{
#pragma unroll
    for (int s = RP_NB / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int q = 0; q < s; ++q) {
            const float send = up ? vals[q] : vals[q + s];
            const float keep = up ? vals[q + s] : vals[q];
            vals[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return vals[0];
}

// Shared memory (offsets in floats).  The column loop's buffers (red .. tauv) alias the
// staged columns Sc, which are dead once the rows are in registers; the exchange buffer
// xbuf, which other ranks write into from column 0 on, aliases nothing.
struct RpLayout {
    int lds;          // row stride of the column-major staging (= rows per CTA)
    bool fused;
    __host__ __device__ RpLayout(int nt, bool f) : lds(nt), fused(f) {}
    // column loop
    __host__ __device__ size_t red() const { return 0; }                     // [32 warps][33]
    __host__ __device__ size_t wsm() const { return 32 * 33 + 4; }           // [32 warps][32], 16-byte
    __host__ __device__ size_t pd() const { return wsm() + 32 * 32; }        // [2][32] pivot row
    __host__ __device__ size_t part() const { return pd() + 64; }            // [2][32] CTA sums
    __host__ __device__ size_t G() const { return part() + 64; }             // [32][RP_GLD]
    __host__ __device__ size_t tauv() const { return G() + 32 * RP_GLD; }    // [32]
    __host__ __device__ size_t loop_end() const { return tauv() + 32; }
    // fused prologue: staged C and V (column-major, stride lds), then small buffers
    __host__ __device__ size_t Sc() const { return 0; }
    __host__ __device__ size_t SVc() const { return (size_t)32 * lds; }
    __host__ __device__ size_t small() const
    {
        const size_t a = fused ? (size_t)64 * lds : 0;
        return ((a > loop_end() ? a : loop_end()) + 3) & ~(size_t)3;
    }
    __host__ __device__ size_t Yp() const { return small(); }                // [32][32]
    __host__ __device__ size_t RS() const { return Yp() + 1024; }            // [48][32]
    __host__ __device__ size_t YS() const { return RS() + 48 * 32; }         // [32][32]
    __host__ __device__ size_t YF() const { return YS() + 1024; }            // [32][32]
    __host__ __device__ size_t Zs() const { return YF() + 1024; }            // [32][32]
    __host__ __device__ size_t Tp() const { return Zs() + 1024; }            // T(q, l) at q + 32 l
    __host__ __device__ size_t CT() const { return Tp() + 1024; }            // [32][33] rank 0
    __host__ __device__ size_t VT() const { return CT() + 32 * 33; }         // [32][33] rank 0
    __host__ __device__ size_t xbuf() const
    {
        const size_t a = fused ? VT() + 32 * 33 : small();
        return (a + 3) & ~(size_t)3;
    }                                                                         // [2][17][RP_XLD]
    __host__ __device__ size_t bytes() const { return sizeof(float) * (xbuf() + 2 * (RP_CL_MAX + 1) * RP_XLD); }
};

}  // namespace

namespace {

// Y = V^T C of this CTA's rows (and, on rank 0, of the 32 rows kp.. above the panel),
// summed over the cluster: every rank ends with the same Y in YF.  Thread tiles of
// 4 (Y rows) x 8 (Y columns) over 8 row groups; the group sum by shuffles.
template <int RPT>
__device__ __forceinline__ void rp_prev_y(const RpLayout &L, float *sm, int rank, int CL, int *flag,
                                          uint64_t *ybar, volatile int *s_abort)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int NT = blockDim.x, lds = L.lds;
    const float *Sc = sm + L.Sc(), *SVc = sm + L.SVc();
    const float *CT = sm + L.CT(), *VT = sm + L.VT();
    float *Yp = sm + L.Yp(), *RS = sm + L.RS(), *YS = sm + L.YS(), *YF = sm + L.YF();
    const int rg = threadIdx.x & 7, slot = threadIdx.x >> 3, nslots = NT >> 3;
    const int rounds = (32 + nslots - 1) / nslots;         // uniform over the CTA
    for (int rd = 0; rd < rounds; ++rd) {
        const int blk = slot + rd * nslots;
        const bool ok = blk < 32;
        const int lb = (blk >> 2) & 7, cb = blk & 3;        // Y rows 4 lb.., Y columns 8 cb..
        float y[4][8];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) y[a][b] = 0.f;
        if (ok) {
            for (int r0 = 4 * rg; r0 < lds; r0 += 32) {     // rows r0 .. r0 + 3
                float4 vq[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) vq[a] = *reinterpret_cast<const float4 *>(SVc + (4 * lb + a) * lds + r0);
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const float4 c4 = *reinterpret_cast<const float4 *>(Sc + (8 * cb + b) * lds + r0);
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        float t = y[a][b];
                        t = fmaf(vq[a].x, c4.x, t);
                        t = fmaf(vq[a].y, c4.y, t);
                        t = fmaf(vq[a].z, c4.z, t);
                        t = fmaf(vq[a].w, c4.w, t);
                        y[a][b] = t;
                    }
                }
            }
            if (rank == 0)
                for (int i = rg; i < 32; i += 8)            // the rows above the panel
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float va = VT[i * 33 + 4 * lb + a];
#pragma unroll
                        for (int b = 0; b < 8; ++b) y[a][b] = fmaf(va, CT[i * 33 + 8 * cb + b], y[a][b]);
                    }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) y[a][b] += __shfl_xor_sync(FULL, y[a][b], o);
        if (ok && rg == 0)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) Yp[(4 * lb + a) * 32 + 8 * cb + b] = y[a][b];
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    // reduce-scatter: row r of the partial goes to rank r % CL, which adds the CL
    // partials in rank order
    const int rpo = (32 + CL - 1) / CL;
    const int mine = (32 - rank + CL - 1) / CL;
    if (threadIdx.x == 0) rp_expect_tx(&ybar[0], (uint32_t)(mine * CL * 128));
    if (threadIdx.x < 32) {
        const int row = threadIdx.x, q = row % CL;
        rp_bulk_to_rank(rp_map(RS + (rank * rpo + row / CL) * 32, q), Yp + row * 32, 128, rp_map(&ybar[0], q));
    }
    if (!tc::mbar_wait(&ybar[0], 0u, RP_SPIN)) {
        *s_abort = 1;
        atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
    }
    for (int idx = threadIdx.x; idx < mine * 32; idx += NT) {
        const int lr = idx / 32, c = idx % 32;
        float sum = 0.f;
        for (int src = 0; src < CL; ++src) sum += RS[(src * rpo + lr) * 32 + c];
        YS[lr * 32 + c] = sum;
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    // all-gather of the summed rows
    if (threadIdx.x == 0) rp_expect_tx(&ybar[1], 32u * 128u);
    for (int idx = threadIdx.x; idx < mine * CL; idx += NT) {
        const int lr = idx / CL, q = idx % CL, row = lr * CL + rank;
        rp_bulk_to_rank(rp_map(YF + row * 32, q), YS + lr * 32, 128, rp_map(&ybar[1], q));
    }
    if (!tc::mbar_wait(&ybar[1], 0u, RP_SPIN)) {
        *s_abort = 1;
        atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
    }
    // Z = T^T Y  (T upper triangular, T(p, q) at Tp[p + 32 q])
    const float *Tp = sm + L.Tp();
    float *Zs = sm + L.Zs();
    for (int idx = threadIdx.x; idx < 1024; idx += NT) {
        const int q = idx / 32, l = idx % 32;
        float z = 0.f;
        for (int p = 0; p <= q; ++p) z = fmaf(Tp[p + 32 * q], YF[p * 32 + l], z);
        Zs[q * 32 + l] = z;
    }
    __syncthreads();
}

// c -= V(row, :) Z for the thread's rows (row t + h NT) held in registers; V(row, :)
// from the staged columns; each row of Z is read once for all the thread's rows
template <int RPT>
__device__ __forceinline__ void rp_apply_rows(const float *SVc, int lds, int NT, const float *Zs,
                                              float (&c)[RPT][RP_NB])
{
#pragma unroll 2
    for (int q = 0; q < RP_NB; ++q) {
        float v[RPT];
#pragma unroll
        for (int h = 0; h < RPT; ++h) v[h] = SVc[q * lds + threadIdx.x + h * NT];
#pragma unroll
        for (int l4 = 0; l4 < 8; ++l4) {
            const float4 z = *reinterpret_cast<const float4 *>(Zs + q * 32 + 4 * l4);
#pragma unroll
            for (int h = 0; h < RPT; ++h) {
                c[h][4 * l4 + 0] = fmaf(-v[h], z.x, c[h][4 * l4 + 0]);
                c[h][4 * l4 + 1] = fmaf(-v[h], z.y, c[h][4 * l4 + 1]);
                c[h][4 * l4 + 2] = fmaf(-v[h], z.z, c[h][4 * l4 + 2]);
                c[h][4 * l4 + 3] = fmaf(-v[h], z.w, c[h][4 * l4 + 3]);
            }
        }
    }
}

}  // namespace

namespace {

// Rows of thread t: t + h NT (h < RPT), panel rows c0 + t + h NT.  One row per thread
// only for CTAs of at most 64 rows (see rp_shape).
template <int RPT>
__global__ void __launch_bounds__(RPT == 1 ? 64 : RP_MAX_ROWS / 2, 1)
k_panel_row(float *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols,
            float *__restrict__ tau_out, float *__restrict__ T_out, int *flag,
            int64_t kp, const float *__restrict__ Tprev)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) float sm[];
    __shared__ uint64_t xbar[2];
    __shared__ uint64_t ybar[2];
    __shared__ uint64_t lbar;                        // bulk loads of the staged columns
    __shared__ volatile int s_abort;

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int NT = blockDim.x, nwarps = NT >> 5;
    const int rpc = RPT * NT;                        // rows per CTA
    const bool fused = kp >= 0;
    const RpLayout L(rpc, fused);
    const int64_t M = m - k;                         // panel rows
    const int64_t c0 = (int64_t)rank * rpc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t g[RPT];
    bool live[RPT];
#pragma unroll
    for (int h = 0; h < RPT; ++h) {
        g[h] = c0 + threadIdx.x + h * NT;
        live[h] = g[h] < M;
    }

    if (threadIdx.x == 0) {
        tc::mbar_init(&xbar[0], 1);
        tc::mbar_init(&xbar[1], 1);
        tc::mbar_init(&ybar[0], 1);
        tc::mbar_init(&ybar[1], 1);
        tc::mbar_init(&lbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();                                 // the bulk loads' barrier is initialised

    // the rows, in registers: loaded straight from F (a warp reads 128 contiguous bytes
    // of each column) or, with the fused update, from the staged columns after it;
    // columns past the panel and rows past the matrix are zero
    float a[RPT][RP_NB];
    if (!fused) {
#pragma unroll
        for (int h = 0; h < RPT; ++h)
#pragma unroll
            for (int l = 0; l < RP_NB; ++l)
                a[h][l] = (live[h] && l < ncols) ? F[(k + g[h]) + (k + l) * ld] : 0.f;
    }

    if (fused) {
        // this panel's columns (C) and the previous panel's reflectors (V) on the CTA's
        // rows, staged column-major by bulk copies of each column's rows.  The factor's
        // rows are padded with zeros to a multiple of 4 (the copies' 16-byte granule);
        // the staged rows past those and C's columns past the panel are zeroed here.
        float *Sc = sm + L.Sc(), *SVc = sm + L.SVc();
        const int nown = (int)fl_max64(0, fl_min64(rpc, M - c0));
        const int nrow4 = (nown + 3) & ~3;
        if (threadIdx.x == 0) {
            const uint32_t bytes = (uint32_t)nrow4 * 4u;
            rp_expect_tx(&lbar, bytes * (uint32_t)(ncols + RP_NB));
            if (nrow4 > 0) {
                for (int l = 0; l < ncols; ++l) rp_bulk_load(Sc + l * rpc, F + (k + c0) + (k + l) * ld, bytes, &lbar);
                for (int q = 0; q < RP_NB; ++q) rp_bulk_load(SVc + q * rpc, F + (k + c0) + (kp + q) * ld, bytes, &lbar);
            }
        }
        for (int idx = threadIdx.x; idx < RP_NB * (rpc - nrow4); idx += NT) {
            const int l = idx / (rpc - nrow4), r = nrow4 + idx % (rpc - nrow4);
            Sc[l * rpc + r] = 0.f;
            SVc[l * rpc + r] = 0.f;
        }
        for (int idx = threadIdx.x; idx < (RP_NB - ncols) * nrow4; idx += NT)
            Sc[(ncols + idx / nrow4) * rpc + idx % nrow4] = 0.f;
        float *Tp = sm + L.Tp();
        for (int idx = threadIdx.x; idx < 1024; idx += NT) Tp[idx] = Tprev[idx];
        if (rank == 0) {
            // rows kp .. kp + 31: this panel's columns (CT) and the previous panel's unit
            // lower triangle (VT)
            float *CT = sm + L.CT(), *VT = sm + L.VT();
            for (int idx = threadIdx.x; idx < 1024; idx += NT) {
                const int i = idx % 32, c = idx / 32;
                CT[i * 33 + c] = (c < ncols) ? F[(kp + i) + (k + c) * ld] : 0.f;
                VT[i * 33 + c] = (i > c) ? F[(kp + i) + (kp + c) * ld] : ((i == c) ? 1.f : 0.f);
            }
        }
    }
    if (fused && !tc::mbar_wait(&lbar, 0u, RP_SPIN)) {
        s_abort = 1;
        atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
    }
    cluster.sync();                                  // barriers ready before any remote signal;
                                                     // staged data visible to the CTA
    if (fused) {
        rp_prev_y<RPT>(L, sm, rank, CL, flag, ybar, &s_abort);
        const float *Sc = sm + L.Sc(), *SVc = sm + L.SVc(), *Zs = sm + L.Zs();
#pragma unroll
        for (int h = 0; h < RPT; ++h)
#pragma unroll
            for (int l = 0; l < RP_NB; ++l) a[h][l] = Sc[l * rpc + threadIdx.x + h * NT];
        rp_apply_rows<RPT>(SVc, rpc, NT, Zs, a);
        if (rank == 0) {
            const float *CT = sm + L.CT(), *VT = sm + L.VT();
            for (int idx = threadIdx.x; idx < 1024; idx += NT) {
                const int i = idx % 32, c = idx / 32;
                float u = 0.f;
                for (int q = 0; q < 32; ++q) u = fmaf(VT[i * 33 + q], Zs[q * 32 + c], u);
                if (c < ncols) F[(kp + i) + (k + c) * ld] = CT[i * 33 + c] - u;
            }
        }
        __syncthreads();                             // staged columns dead from here on
    }

    float *red = sm + L.red(), *wsm = sm + L.wsm(), *pd = sm + L.pd(), *part = sm + L.part();
    float *G = sm + L.G(), *tauv = sm + L.tauv(), *xbuf = sm + L.xbuf();
    for (int idx = threadIdx.x; idx < 32 * RP_GLD; idx += NT) G[idx] = 0.f;
    if (threadIdx.x < 32) tauv[threadIdx.x] = 0.f;
    const uint32_t xbytes = (uint32_t)(CL + 1) * 32u * (uint32_t)sizeof(float);

    // (a loop, not unrolled: 32 unrolled steps do not fit in the instruction caches;
    // the register column j is picked by selects)
#pragma unroll 1
    for (int j = 0; j < ncols; ++j) {
        const int par = j & 1;
        float *xb = xbuf + par * (RP_CL_MAX + 1) * RP_XLD;
        if (threadIdx.x == 0) rp_expect_tx(&xbar[par], xbytes);
        {
            // products a_j a_l of the rows below the pivot, summed over the thread's rows,
            // then over the warp
            float P[RP_NB];
#pragma unroll
            for (int l = 0; l < RP_NB; ++l) P[l] = 0.f;
#pragma unroll
            for (int h = 0; h < RPT; ++h) {
                float ajx = 0.f;
#pragma unroll
                for (int l = 0; l < RP_NB; ++l) ajx = (l == j) ? a[h][l] : ajx;
                const float aj = (live[h] && g[h] > j) ? ajx : 0.f;
#pragma unroll
                for (int l = 0; l < RP_NB; ++l) P[l] = fmaf(aj, a[h][l], P[l]);
            }
            red[warp * 33 + lane] = rp_reduce_scatter(P, lane);
        }
        if (g[0] == j) {                             // rank 0, thread j: the pivot row
#pragma unroll
            for (int l = 0; l < RP_NB; ++l) pd[par * 32 + l] = a[0][l];
        }
        __syncthreads();
        if (s_abort) break;                          // uniform after the barrier
        if (warp == 0) {
            float s0 = 0.f, s1 = 0.f;
            int w = 0;
            for (; w + 1 < nwarps; w += 2) {
                s0 += red[w * 33 + lane];
                s1 += red[(w + 1) * 33 + lane];
            }
            if (w < nwarps) s0 += red[w * 33 + lane];
            part[par * 32 + lane] = s0 + s1;
            __syncwarp();
            // 16-byte pieces: the CTA's sums to every rank, and rank 0's pivot row
            for (int idx = lane; idx < CL * 8; idx += 32) {
                const int q = idx >> 3, i = idx & 7;
                const uint32_t rb = rp_map(&xbar[par], q);
                rp_st_async_v4(rp_map(xb + rank * RP_XLD + 4 * i, q),
                               *reinterpret_cast<const float4 *>(part + par * 32 + 4 * i), rb);
                if (rank == 0)
                    rp_st_async_v4(rp_map(xb + RP_CL_MAX * RP_XLD + 4 * i, q),
                                   *reinterpret_cast<const float4 *>(pd + par * 32 + 4 * i), rb);
            }
        }
        if (!tc::mbar_wait(&xbar[par], (uint32_t)(j >> 1) & 1u, RP_SPIN)) {
            s_abort = 1;                             // every warp leaves at the next barrier
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        }
        // every warp adds the ranks' sums in the same order: identical scalars everywhere
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
        for (int q = 0; q < RP_CL_MAX; q += 4) {
            if (q < CL) d0 += xb[q * RP_XLD + lane];
            if (q + 1 < CL) d1 += xb[(q + 1) * RP_XLD + lane];
            if (q + 2 < CL) d2 += xb[(q + 2) * RP_XLD + lane];
            if (q + 3 < CL) d3 += xb[(q + 3) * RP_XLD + lane];
        }
        const float dl = (d0 + d1) + (d2 + d3);
        const float ss = __shfl_sync(FULL, dl, j);
        const float alpha = xb[RP_CL_MAX * RP_XLD + j];
        const float pl = xb[RP_CL_MAX * RP_XLD + lane];
        float beta = alpha, tj = 0.f, inv = 0.f;
        if (!isfinite(ss) || !isfinite(alpha)) {
            if (threadIdx.x == 0) atomicCAS(flag, 0, FL_DEVERR_NONFINITE);
        } else if (ss > 0.f) {
            // reflector of column j: v = 1 at row j, a(j+1:)/(a_jj - beta) below
            const float nrm = sqrtf(alpha * alpha + ss);
            beta = (alpha >= 0.f) ? -nrm : nrm;
            tj = __fdividef(beta - alpha, beta);     // |beta| >= |alpha| > 0: in range, 2 ulp
            inv = __fdividef(1.f, alpha - beta);
        }
        if (rank == 0 && warp == 0) {
            if (lane < j) G[lane * RP_GLD + j] = fmaf(inv, dl, pl);   // v_l^T v_j
            if (lane == 0) tauv[j] = tj;
        }
        wsm[warp * 32 + lane] = (lane > j) ? tj * fmaf(inv, dl, pl) : 0.f;
        __syncwarp();
        float w[RP_NB];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 t = *reinterpret_cast<const float4 *>(wsm + warp * 32 + 4 * i);
            w[4 * i] = t.x;
            w[4 * i + 1] = t.y;
            w[4 * i + 2] = t.z;
            w[4 * i + 3] = t.w;
        }
        // rows below the pivot: v = a_j inv into column j, a_l -= w_l v; the pivot row:
        // beta into column j, a_l -= w_l; rows above: unchanged (w_l = 0 for l <= j)
#pragma unroll
        for (int h = 0; h < RPT; ++h) {
            const bool below = live[h] && g[h] > j, piv = g[h] == j;
            float ajx = 0.f;
#pragma unroll
            for (int l = 0; l < RP_NB; ++l) ajx = (l == j) ? a[h][l] : ajx;
            const float v = ajx * inv;
            const float vv = below ? v : (piv ? 1.f : 0.f);
            const float nj = below ? v : (piv ? beta : ajx);
#pragma unroll
            for (int l = 0; l < RP_NB; ++l) a[h][l] = (l == j) ? nj : fmaf(-w[l], vv, a[h][l]);
        }
    }

    // the factored rows: R on and above the diagonal, V below
    {
        // (the base pointer is opaque here, so that the column addresses of the loads
        // above are not kept live through the column loop for reuse)
        float *Fo = F;
        int64_t ldo = ld;
        asm volatile("" : "+l"(Fo), "+l"(ldo));
#pragma unroll
        for (int h = 0; h < RPT; ++h)
            if (live[h]) {
                float *dst = Fo + (k + g[h]) + k * ldo;
#pragma unroll
                for (int l = 0; l < RP_NB; ++l)
                    if (l < ncols) dst[l * ldo] = a[h][l];
            }
    }
    if (rank == 0 && warp == 0) {
        // T = (I + D N)^{-1} D with N = striu(V^T V), D = diag(tau): lane c solves the
        // unit upper triangular system for column c by substitution from the bottom
        __syncwarp();
        const int c = lane;
        float x[RP_NB];
#pragma unroll
        for (int i = RP_NB - 1; i >= 0; --i) {
            float acc = 0.f;
#pragma unroll
            for (int q = i + 1; q < RP_NB; ++q) acc = fmaf(G[i * RP_GLD + q], x[q], acc);
            x[i] = ((i == c) ? 1.f : 0.f) - tauv[i] * acc;
        }
        const float tc_ = tauv[c];
#pragma unroll
        for (int i = 0; i < RP_NB; ++i) T_out[i + RP_NB * c] = x[i] * tc_;
        tau_out[lane] = (lane < ncols) ? tauv[lane] : 0.f;
    }
    // no CTA leaves while another may still store into its shared memory
    cluster.sync();
}

}  // namespace

namespace {

template <int RPT>
int launch_panel_row(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols, int CL,
                     int NT, float *tau, float *Tblk, int64_t kp, const float *Tprev)
{
    const RpLayout L(RPT * NT, kp >= 0);
    const size_t smem = L.bytes();
    const size_t cap = (size_t)ctx->max_smem_optin - 1024;          // static shared memory aside
    if (smem > cap) return 2;
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_panel_row<RPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_panel_row<RPT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "cudaFuncSetAttribute");
        attr_once.done(ctx->device);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(NT);
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_panel_row<RPT>, F, ld, k, m_aug, ncols, tau, Tblk, ctx->d_flag,
                                       kp, Tprev);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "row panel launch");
    return 0;
}

// cluster size, rows per thread and threads per CTA for a panel of mp rows;
// false when the panel is too tall (more than 768 rows per CTA)
struct RpShape {
    int CL, RPT, NT;
};

bool rp_shape(int64_t mp, RpShape &s)
{
    // one CTA without any exchange for short panels; otherwise as many CTAs as the
    // cluster allows (the per-column exchange costs about the same for any size)
    s.CL = mp <= RP_MAX_ROWS ? 1 : (int)std::min<int64_t>(RP_CL_MAX, fl_cdiv(mp, 64));
    const int64_t rows = fl_cdiv(mp, s.CL);
    if (rows > RP_MAX_ROWS) return false;
    s.RPT = rows > 64 ? 2 : 1;
    s.NT = (int)fl_round_up(fl_cdiv(rows, s.RPT), 32);
    return true;
}

}  // namespace

// 0 on launch, 1 when the panel is too tall for the row kernel, 2 when the fused form
// does not fit in shared memory (the caller then uses another panel kernel)
int fl_panel_row_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                     float *tau, float *Tblk, int64_t kp, const float *Tprev)
{
    RpShape s;
    if (!rp_shape(m_aug - k, s)) return 1;
    if (s.RPT == 2) return launch_panel_row<2>(ctx, F, ld, k, m_aug, ncols, s.CL, s.NT, tau, Tblk, kp, Tprev);
    return launch_panel_row<1>(ctx, F, ld, k, m_aug, ncols, s.CL, s.NT, tau, Tblk, kp, Tprev);
}

bool fl_panel_row_fits(fastlsq_ctx *ctx, int64_t mp, bool fused)
{
    RpShape s;
    if (!rp_shape(mp, s)) return false;
    return RpLayout(s.RPT * s.NT, fused).bytes() <= (size_t)ctx->max_smem_optin - 1024;
}

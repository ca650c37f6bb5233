// Tall-panel factorisation for the FP32 factor (panel width 16, more rows than the
// register panels hold): Householder QR of the panel (Sec. 2.3, LAPACK sign
// convention, compact-WY T) on a cluster of up to 16 CTAs.
//
// CTA c holds panel rows [c * rpc, (c + 1) * rpc) in shared memory, one 16-float row
// per 80 bytes (16-byte loads of a row by consecutive threads are conflict-free);
// thread t works on rows t, t + 768, ...  The 16 column steps are unrolled (the
// column index is a constant in each), and one pass over the rows per column both
// applies H_j and forms the products a_{j+1} a_l (l = 0 .. 15, rows below j + 1) that
// the next step needs:
//   * l > j + 1: the dots of the next pivot column with the columns right of it;
//   * l = j + 1: the squared norm below the next pivot;
//   * l < j + 1: with the pivot row and 1 / (a_jj - beta), the Gram entries
//     v_l^T v_{j+1} of the reflectors, from which T = (I + D striu(V^T V))^{-1} D,
//     D = diag(tau), is formed at the end (one lane per column of T).
// Per column the warps' sums are added in a fixed order, the CTA's 16 sums and, on
// rank 0, the pivot row go to every rank as asynchronous DSMEM stores that count down
// the receiver's barrier, and every warp adds the ranks' sums in the same order, so
// all threads of all ranks hold bit-identical reflector scalars.  Waits are bounded
// (about a second of SM clock): on timeout the device flag is raised and the
// remaining steps are skipped.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "qr.cuh"
#include "tc_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int PT_NB = 16;
constexpr int PT_CL = 16;                      // CTAs per cluster (at most)
constexpr int PT_NT = 768;                     // threads per CTA
constexpr int PT_NW = PT_NT / 32;
constexpr int PT_LD = 20;                      // row stride in floats (80 bytes)
constexpr int PT_MAX_RPC = 2816;               // rows per CTA
constexpr int64_t PT_MIN_ROWS = 4096;          // shorter panels use the register kernels
constexpr long long PT_SPIN = 2000000000ll;    // SM cycles (about a second) before a wait gives up

__device__ __forceinline__ uint32_t pt_map(const void *p, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(tc::smem_addr(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void pt_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void pt_st_async_v4(uint32_t addr, float4 v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];\n"
                 :: "r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar) : "memory");
}

// lanes l and l + 16 return the warp's sum of v[l] (16 shuffles; v is overwritten)
__device__ __forceinline__ float pt_reduce16(float (&v)[PT_NB], int lane)
{
#pragma unroll
    for (int s = PT_NB / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int q = 0; q < s; ++q) {
            const float send = up ? v[q] : v[q + s];
            const float keep = up ? v[q + s] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

__device__ __forceinline__ void pt_load_row(const float *row, float (&a)[PT_NB])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 t = *reinterpret_cast<const float4 *>(row + 4 * q);
        a[4 * q] = t.x;
        a[4 * q + 1] = t.y;
        a[4 * q + 2] = t.z;
        a[4 * q + 3] = t.w;
    }
}

// Shared memory (offsets in floats; every piece starts on 16 bytes)
struct PtLayout {
    int rpc;
    __host__ __device__ explicit PtLayout(int r) : rpc(r) {}
    __host__ __device__ size_t P() const { return 0; }                                 // [rpc][PT_LD]
    __host__ __device__ size_t xbuf() const { return (size_t)rpc * PT_LD; }            // [2][PT_CL + 1][PT_LD]
    __host__ __device__ size_t red() const { return xbuf() + 2 * (PT_CL + 1) * PT_LD; } // [PT_NW][17] (+ pad)
    __host__ __device__ size_t part() const { return red() + ((PT_NW * 17 + 3) & ~3); } // [2][16]
    __host__ __device__ size_t pd() const { return part() + 32; }                      // [2][16] pivot rows
    __host__ __device__ size_t G() const { return pd() + 32; }                         // [16][17]
    __host__ __device__ size_t tauv() const { return G() + ((16 * 17 + 3) & ~3); }     // [16]
    __host__ __device__ size_t loop_end() const { return tauv() + 16; }
    // the fused prologue (the previous panel's update of this panel's columns)
    __host__ __device__ size_t Yst() const { return loop_end(); }                     // [PT_NW][256]
    __host__ __device__ size_t Yc() const { return Yst() + PT_NW * 256; }              // [256] CTA sums
    __host__ __device__ size_t YR() const { return Yc() + 256; }                       // [CL][16 / CL][16]
    __host__ __device__ size_t Yf() const { return YR() + 256; }                       // [16][16] Y
    __host__ __device__ size_t Zs() const { return Yf() + 256; }                       // [16][16] Z
    __host__ __device__ size_t Tp() const { return Zs() + 256; }                       // T(q, l) at q + 16 l
    __host__ __device__ size_t CT() const { return Tp() + 256; }                       // [16][17] rank 0
    __host__ __device__ size_t VT() const { return CT() + 16 * 17; }                   // [16][17] rank 0
    __host__ __device__ size_t bytes(bool fused) const
    {
        return sizeof(float) * (fused ? VT() + 16 * 17 : loop_end());
    }
};

}  // namespace

namespace {

// The previous panel's update of this panel's columns (its reflectors V_p at columns
// kp.., its T_p): C -= V_p T_p^T V_p^T C on rows kp.. of this panel's columns.  Y =
// V_p^T C by warps over the CTA's rows (lane: column l of V_p, 8 columns of C), summed
// over the warps in a fixed order, then over the cluster by a reduce-scatter (rank q
// adds rows l = q mod CL of Y in rank order) and an all-gather; Z = T_p^T Y; then each
// thread updates its rows in shared memory.  Rank 0 also takes the 16 rows kp.. above
// the panel (V_p's unit lower triangle there) and writes them back.  False when a
// wait ran out.
__device__ __forceinline__ bool pt_prologue(const PtLayout &L, float *sm, float *__restrict__ F, int64_t ld,
                                            int64_t k, int64_t kp, int64_t c0, int nown, int rank, int CL,
                                            int ncols, uint64_t *ybar)
{
    float *P = sm + L.P(), *Yst = sm + L.Yst(), *Yc = sm + L.Yc(), *YR = sm + L.YR(), *Yf = sm + L.Yf();
    float *Zs = sm + L.Zs();
    const float *Tp = sm + L.Tp(), *CT = sm + L.CT(), *VT = sm + L.VT();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *Vp = F + (k + c0) + kp * ld;        // V_p(panel row r of this CTA, l) at Vp[r + l ld]
    {
        // warp w takes rows [r0, r1) in chunks of 16: the chunk of V_p is staged in the
        // warp's slice of Yst by 16-byte loads along F's columns (rows start on 16 bytes:
        // k and the CTA's first row are multiples of 4), then lane (l, h) adds
        // V_p(r, l) C(r, 8h .. 8h + 7) over the chunk's rows
        const int l = lane & 15, h = lane >> 4;
        const int rw = ((nown + PT_NW - 1) / PT_NW + 15) & ~15;
        const int r0 = warp * rw, r1 = min(nown, r0 + rw);
        float *Vst = Yst + warp * 256;                   // [16 rows][16]
        float y[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) y[e] = 0.f;
        const int lc = lane >> 1, lh = lane & 1;          // staging: column lc, rows 8 lh .. 8 lh + 7
        for (int rc = r0; rc < r1; rc += 16) {
            const float *src = Vp + (rc + 8 * lh) + lc * ld;
            const float4 u0 = (rc + 8 * lh < r1) ? __ldg(reinterpret_cast<const float4 *>(src))
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 u1 = (rc + 8 * lh + 4 < r1) ? __ldg(reinterpret_cast<const float4 *>(src + 4))
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
            const float uv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j)
                Vst[(8 * lh + j) * 16 + lc] = (rc + 8 * lh + j < r1) ? uv[j] : 0.f;
            __syncwarp();
            const int nr = min(16, r1 - rc);
            for (int i = 0; i < nr; ++i) {
                const float v = Vst[i * 16 + l];
                const float *prow = P + (rc + i) * PT_LD + 8 * h;
                const float4 a = *reinterpret_cast<const float4 *>(prow);
                const float4 b = *reinterpret_cast<const float4 *>(prow + 4);
                y[0] = fmaf(v, a.x, y[0]);
                y[1] = fmaf(v, a.y, y[1]);
                y[2] = fmaf(v, a.z, y[2]);
                y[3] = fmaf(v, a.w, y[3]);
                y[4] = fmaf(v, b.x, y[4]);
                y[5] = fmaf(v, b.y, y[5]);
                y[6] = fmaf(v, b.z, y[6]);
                y[7] = fmaf(v, b.w, y[7]);
            }
        }
        __syncwarp();
        float *dst = Yst + warp * 256 + l * 16 + 8 * h;
        *reinterpret_cast<float4 *>(dst) = make_float4(y[0], y[1], y[2], y[3]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(y[4], y[5], y[6], y[7]);
    }
    __syncthreads();
    if (threadIdx.x < 256) {
        const int t = threadIdx.x;
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int w = 0; w < PT_NW; w += 2) {
            s0 += Yst[w * 256 + t];
            s1 += Yst[(w + 1) * 256 + t];
        }
        float s = s0 + s1;
        if (rank == 0) {                               // rows kp .. kp + 15
            const int l = t >> 4, c = t & 15;
            float u = 0.f;
#pragma unroll
            for (int i = 0; i < 16; ++i) u = fmaf(VT[i * 17 + l], CT[i * 17 + c], u);
            s += u;
        }
        Yc[t] = s;
    }
    __syncthreads();
    // reduce-scatter: row l of the CTA's sums to rank l mod CL, in 16-byte pieces
    const int rpr = PT_NB / CL;                        // rows of Y per rank
    if (threadIdx.x == 0) pt_expect_tx(&ybar[0], (uint32_t)(CL * rpr * 64));
    if (threadIdx.x < 64) {
        const int l = threadIdx.x >> 2, c4 = threadIdx.x & 3, q = l % CL, j = l / CL;
        pt_st_async_v4(pt_map(YR + (rank * rpr + j) * 16 + 4 * c4, q),
                       *reinterpret_cast<const float4 *>(Yc + l * 16 + 4 * c4), pt_map(&ybar[0], q));
    }
    bool ok = tc::mbar_wait(&ybar[0], 0u, PT_SPIN);
    // the rank's rows of Y, added over the ranks in rank order, to every rank
    if (threadIdx.x == 0) pt_expect_tx(&ybar[1], (uint32_t)(PT_NB * 64));
    if (threadIdx.x < rpr * 4) {
        const int j = threadIdx.x >> 2, c4 = threadIdx.x & 3, l = rank + j * CL;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int src = 0; src < CL; ++src) {
            const float4 v = *reinterpret_cast<const float4 *>(YR + (src * rpr + j) * 16 + 4 * c4);
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        for (int q = 0; q < CL; ++q) pt_st_async_v4(pt_map(Yf + l * 16 + 4 * c4, q), acc, pt_map(&ybar[1], q));
    }
    ok = tc::mbar_wait(&ybar[1], 0u, PT_SPIN) && ok;
    // Z = T_p^T Y  (T_p upper triangular)
    if (threadIdx.x < 256) {
        const int q = threadIdx.x >> 4, c = threadIdx.x & 15;
        float z = 0.f;
        for (int p = 0; p <= q; ++p) z = fmaf(Tp[p + 16 * q], Yf[p * 16 + c], z);
        Zs[q * 16 + c] = z;
    }
    __syncthreads();
    // C -= V_p Z on the CTA's rows, two rows per thread at a time (Z's rows are read once
    // for both)
    for (int r = threadIdx.x; r < nown; r += 2 * PT_NT) {
        const int r2 = r + PT_NT;
        const bool two = r2 < nown;
        float c[2][PT_NB];
        pt_load_row(P + r * PT_LD, c[0]);
        pt_load_row(P + (two ? r2 : r) * PT_LD, c[1]);
#pragma unroll 4
        for (int l = 0; l < PT_NB; ++l) {
            const float v0 = __ldg(Vp + r + l * ld);
            const float v1 = two ? __ldg(Vp + r2 + l * ld) : 0.f;
            float z[PT_NB];
            pt_load_row(Zs + l * 16, z);
#pragma unroll
            for (int cc = 0; cc < PT_NB; ++cc) {
                c[0][cc] = fmaf(-v0, z[cc], c[0][cc]);
                c[1][cc] = fmaf(-v1, z[cc], c[1][cc]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            *reinterpret_cast<float4 *>(P + r * PT_LD + 4 * q) =
                make_float4(c[0][4 * q], c[0][4 * q + 1], c[0][4 * q + 2], c[0][4 * q + 3]);
            if (two)
                *reinterpret_cast<float4 *>(P + r2 * PT_LD + 4 * q) =
                    make_float4(c[1][4 * q], c[1][4 * q + 1], c[1][4 * q + 2], c[1][4 * q + 3]);
        }
    }
    if (rank == 0 && threadIdx.x < 256) {              // rows kp .. kp + 15, final
        const int i = threadIdx.x >> 4, c = threadIdx.x & 15;
        float u = 0.f;
#pragma unroll
        for (int q = 0; q < 16; ++q) u = fmaf(VT[i * 17 + q], Zs[q * 16 + c], u);
        if (c < ncols) F[(kp + i) + (k + c) * ld] = CT[i * 17 + c] - u;
    }
    __syncthreads();
    return ok;
}

template <bool FUSED>
__global__ void __launch_bounds__(PT_NT, 1)
k_panel_tall(float *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols, int rpc,
             float *__restrict__ tau_out, float *__restrict__ T_out, int *flag, int64_t kp,
             const float *__restrict__ Tprev)
{
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) float sm[];
    __shared__ uint64_t xbar[2];
    __shared__ uint64_t ybar[2];
    __shared__ volatile int s_abort;

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const PtLayout L(rpc);
    float *P = sm + L.P(), *xbuf = sm + L.xbuf(), *red = sm + L.red(), *part = sm + L.part();
    float *pd = sm + L.pd(), *G = sm + L.G(), *tauv = sm + L.tauv();
    const int64_t M = m - k;                          // panel rows
    const int64_t c0 = (int64_t)rank * rpc;
    const int nown = (int)fl_max64(0, fl_min64(rpc, M - c0));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, cl = lane & 15;

    if (threadIdx.x == 0) {
        tc::mbar_init(&xbar[0], 1);
        tc::mbar_init(&xbar[1], 1);
        tc::mbar_init(&ybar[0], 1);
        tc::mbar_init(&ybar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    // the CTA's rows (columns past the panel zero), read along F's columns: a thread's
    // rows r, r + 768, .. of all 16 columns, their loads in flight together, then each
    // row as 16-byte stores
    for (int r0 = threadIdx.x; r0 < nown; r0 += 2 * PT_NT) {
        float a[2][PT_NB];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + h * PT_NT;
#pragma unroll
            for (int c = 0; c < PT_NB; ++c)
                a[h][c] = (r < nown && c < ncols) ? F[(k + c0 + r) + (k + c) * ld] : 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + h * PT_NT;
            if (r < nown)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<float4 *>(P + r * PT_LD + 4 * q) =
                        make_float4(a[h][4 * q], a[h][4 * q + 1], a[h][4 * q + 2], a[h][4 * q + 3]);
        }
    }
    for (int idx = threadIdx.x; idx < 16 * 17; idx += PT_NT) G[idx] = 0.f;
    if (threadIdx.x < 16) tauv[threadIdx.x] = 0.f;
    if constexpr (FUSED) {
        float *Tp = sm + L.Tp(), *CT = sm + L.CT(), *VT = sm + L.VT();
        for (int idx = threadIdx.x; idx < 256; idx += PT_NT) Tp[idx] = Tprev[idx];
        if (rank == 0)
            for (int idx = threadIdx.x; idx < 256; idx += PT_NT) {
                // rows kp .. kp + 15: this panel's columns, the previous panel's unit lower triangle
                const int i = idx % 16, c = idx / 16;
                CT[i * 17 + c] = (c < ncols) ? F[(kp + i) + (k + c) * ld] : 0.f;
                VT[i * 17 + c] = (i > c) ? F[(kp + i) + (kp + c) * ld] : ((i == c) ? 1.f : 0.f);
            }
    }
    cluster.sync();      // barriers initialised on every rank before any remote store; rows visible
    if constexpr (FUSED) {
        if (!pt_prologue(L, sm, F, ld, k, kp, c0, nown, rank, CL, ncols, ybar)) {
            s_abort = 1;                               // read by every thread after the next barrier
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        }
    }

    // products of column 0 with every column over the rows below 0; pivot row 0
    float pr[PT_NB];
#pragma unroll
    for (int l = 0; l < PT_NB; ++l) pr[l] = 0.f;
    for (int r = threadIdx.x; r < nown; r += PT_NT) {
        float a[PT_NB];
        pt_load_row(P + r * PT_LD, a);
        if (c0 + r > 0) {
#pragma unroll
            for (int l = 0; l < PT_NB; ++l) pr[l] = fmaf(a[0], a[l], pr[l]);
        } else {
#pragma unroll
            for (int l = 0; l < PT_NB; ++l) pd[l] = a[l];
        }
    }
    const uint32_t xbytes = (uint32_t)(CL + 1) * PT_NB * (uint32_t)sizeof(float);

    auto step = [&](auto jc) {
        constexpr int J = decltype(jc)::value;
        constexpr int par = J & 1;
        if (J >= ncols) return;                       // uniform (a kernel argument)
        float *xb = xbuf + par * (PT_CL + 1) * PT_LD;
        if (threadIdx.x == 0) pt_expect_tx(&xbar[par], xbytes);
        {
            const float s = pt_reduce16(pr, lane);
            if (lane < 16) red[warp * 17 + lane] = s;
        }
        __syncthreads();
        if (s_abort) return;                          // uniform: only set before this barrier
        if (warp == 0) {
            if (lane < 16) {
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int w = 0; w < PT_NW; w += 2) {
                    s0 += red[w * 17 + lane];
                    s1 += red[(w + 1) * 17 + lane];
                }
                part[par * 16 + lane] = s0 + s1;
            }
            __syncwarp();
            // 16-byte pieces: the CTA's sums to every rank, and rank 0's pivot row
            for (int idx = lane; idx < CL * 4; idx += 32) {
                const int q = idx >> 2, i = idx & 3;
                const uint32_t rb = pt_map(&xbar[par], q);
                pt_st_async_v4(pt_map(xb + rank * PT_LD + 4 * i, q),
                               *reinterpret_cast<const float4 *>(part + par * 16 + 4 * i), rb);
                if (rank == 0)
                    pt_st_async_v4(pt_map(xb + PT_CL * PT_LD + 4 * i, q),
                                   *reinterpret_cast<const float4 *>(pd + par * 16 + 4 * i), rb);
            }
        }
        if (!tc::mbar_wait(&xbar[par], (uint32_t)(J >> 1) & 1u, PT_SPIN)) {
            s_abort = 1;                              // every warp leaves after the next barrier
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        }
        // every warp adds the ranks' sums in the same order: identical scalars everywhere
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll
        for (int q = 0; q < PT_CL; q += 4) {
            if (q < CL) d0 += xb[q * PT_LD + cl];
            if (q + 1 < CL) d1 += xb[(q + 1) * PT_LD + cl];
            if (q + 2 < CL) d2 += xb[(q + 2) * PT_LD + cl];
            if (q + 3 < CL) d3 += xb[(q + 3) * PT_LD + cl];
        }
        const float dl = (d0 + d1) + (d2 + d3);
        const float ss = __shfl_sync(FULL, dl, J);
        const float alpha = xb[PT_CL * PT_LD + J];
        const float pl = xb[PT_CL * PT_LD + cl];
        float beta = alpha, tj = 0.f, inv = 0.f;
        if (!isfinite(ss) || !isfinite(alpha)) {
            if (threadIdx.x == 0) atomicCAS(flag, 0, FL_DEVERR_NONFINITE);
        } else if (ss > 0.f) {
            // reflector of column J: v = 1 at row J, a(J+1:)/(a_JJ - beta) below
            const float nrm = sqrtf(alpha * alpha + ss);
            beta = (alpha >= 0.f) ? -nrm : nrm;
            tj = (beta - alpha) / beta;
            inv = 1.f / (alpha - beta);
        }
        if (rank == 0 && warp == 0) {
            if (lane < J) G[lane * 17 + J] = fmaf(inv, dl, pl);       // v_l^T v_J
            if (lane == 0) tauv[J] = tj;
        }
        // w_l = tau v^T a_l for the columns right of the pivot
        const float wl = (cl > J) ? tj * fmaf(inv, dl, pl) : 0.f;
        float w[PT_NB];
#pragma unroll
        for (int l = 0; l < PT_NB; ++l) w[l] = (l > J) ? __shfl_sync(FULL, wl, l) : 0.f;

        // rows below the pivot: v = a_J inv into column J, a_l -= w_l v; the pivot row:
        // beta into column J, a_l -= w_l; rows above: unchanged.  Then the products of
        // the next pivot column (rows below it) and the next pivot row.
        const bool nextp = J + 1 < ncols;
#pragma unroll
        for (int l = 0; l < PT_NB; ++l) pr[l] = 0.f;
        for (int r = threadIdx.x; r < nown; r += PT_NT) {
            const int64_t g = c0 + r;
            if (g < J) continue;
            float *row = P + r * PT_LD;
            float a[PT_NB];
            pt_load_row(row, a);
            if (g > J) {
                const float v = a[J] * inv;
                a[J] = v;
#pragma unroll
                for (int l = J + 1; l < PT_NB; ++l) a[l] = fmaf(-w[l], v, a[l]);
            } else {
                a[J] = beta;
#pragma unroll
                for (int l = J + 1; l < PT_NB; ++l) a[l] -= w[l];
            }
#pragma unroll
            for (int q = J / 4; q < 4; ++q)
                *reinterpret_cast<float4 *>(row + 4 * q) = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
            if constexpr (J + 1 < PT_NB) {
                if (nextp) {
                    if (g > J + 1) {
                        const float an = a[J + 1];
#pragma unroll
                        for (int l = 0; l < PT_NB; ++l) pr[l] = fmaf(an, a[l], pr[l]);
                    } else if (g == J + 1) {
#pragma unroll
                        for (int l = 0; l < PT_NB; ++l) pd[(par ^ 1) * 16 + l] = a[l];
                    }
                }
            }
        }
    };
    step(std::integral_constant<int, 0>{});
    step(std::integral_constant<int, 1>{});
    step(std::integral_constant<int, 2>{});
    step(std::integral_constant<int, 3>{});
    step(std::integral_constant<int, 4>{});
    step(std::integral_constant<int, 5>{});
    step(std::integral_constant<int, 6>{});
    step(std::integral_constant<int, 7>{});
    step(std::integral_constant<int, 8>{});
    step(std::integral_constant<int, 9>{});
    step(std::integral_constant<int, 10>{});
    step(std::integral_constant<int, 11>{});
    step(std::integral_constant<int, 12>{});
    step(std::integral_constant<int, 13>{});
    step(std::integral_constant<int, 14>{});
    step(std::integral_constant<int, 15>{});
    __syncthreads();

    // the factored rows: R on and above the diagonal, V below
    for (int r = threadIdx.x; r < nown; r += PT_NT) {
        float a[PT_NB];
        pt_load_row(P + r * PT_LD, a);
#pragma unroll
        for (int c = 0; c < PT_NB; ++c)
            if (c < ncols) F[(k + c0 + r) + (k + c) * ld] = a[c];
    }
    if (rank == 0 && warp == 0) {
        // T = (I + D N)^{-1} D with N = striu(V^T V), D = diag(tau): lane c solves the
        // unit upper triangular system for column c by substitution from the bottom
        const int c = cl;
        float x[PT_NB];
#pragma unroll
        for (int i = PT_NB - 1; i >= 0; --i) {
            float acc = 0.f;
#pragma unroll
            for (int q = i + 1; q < PT_NB; ++q) acc = fmaf(G[i * 17 + q], x[q], acc);
            x[i] = ((i == c) ? 1.f : 0.f) - tauv[i] * acc;
        }
        if (lane < 16) {
            const float tc_ = tauv[c];
#pragma unroll
            for (int i = 0; i < PT_NB; ++i) T_out[i + PT_NB * c] = x[i] * tc_;
            tau_out[lane] = (lane < ncols) ? tauv[lane] : 0.f;
        }
    }
    // no CTA leaves while another may still store into its shared memory
    cluster.sync();
}

// cluster size and rows per CTA for a panel of mp rows; false when it does not fit
bool pt_shape(int64_t mp, int &CL, int &rpc)
{
    CL = PT_CL;
    while (CL > 1 && fl_cdiv(mp, CL) < PT_NB) CL >>= 1;
    rpc = (int)fl_round_up(std::max<int64_t>(PT_NB, fl_cdiv(mp, CL)), 4);   // CTA rows start on 16 bytes
    return rpc <= PT_MAX_RPC;
}

}  // namespace

bool fl_panel_tall_fits(fastlsq_ctx *ctx, int64_t mp, bool fused)
{
    int CL, rpc;
    if (mp < PT_MIN_ROWS || !pt_shape(mp, CL, rpc)) return false;
    return PtLayout(rpc).bytes(fused) <= (size_t)ctx->max_smem_optin - 1024;
}

namespace {

template <bool FUSED>
int launch_panel_tall(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols, float *tau,
                      float *Tblk, int64_t kp, const float *Tprev)
{
    int CL, rpc;
    if (!fl_panel_tall_fits(ctx, m_aug - k, FUSED) || !pt_shape(m_aug - k, CL, rpc)) return 1;
    const size_t smem = PtLayout(rpc).bytes(FUSED);
    const size_t cap = (size_t)ctx->max_smem_optin - 1024;          // static shared memory aside
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_panel_tall<FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)cap);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_panel_tall<FUSED>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "cudaFuncSetAttribute");
        attr_once.done(ctx->device);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(PT_NT);
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
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_panel_tall<FUSED>, F, ld, k, m_aug, ncols, rpc, tau, Tblk,
                                       ctx->d_flag, kp, Tprev);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "tall panel launch");
    return 0;
}

}  // namespace

int fl_panel_tall_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                      float *tau, float *Tblk, int64_t kp, const float *Tprev)
{
    if (kp >= 0) return launch_panel_tall<true>(ctx, F, ld, k, m_aug, ncols, tau, Tblk, kp, Tprev);
    return launch_panel_tall<false>(ctx, F, ld, k, m_aug, ncols, tau, Tblk, -1, nullptr);
}

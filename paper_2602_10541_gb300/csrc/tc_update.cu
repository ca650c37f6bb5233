// Trailing update of the blocked Householder QR on the tcgen05 tensor cores, in
// split TF32x3 precision with FP32 accumulation in TMEM:
//   x = hi + lo (hi = tf32 rounding of x, lo = x - hi), a*b ~ ah*bh + ah*bl + al*bh.
// For panel k with Householder block V (m_p x 32, unit lower trapezoidal) and
// compact-WY factor T, C -= V (T^T (V^T C)) in two kernels:
//   k_tcy : Y^T = C^T V over interleaved row chunks (MMA M = 128 columns of C, N = 32,
//           K = rows in chunks of 32).  A ring of 3 landing slots is filled by TMA: a C
//           chunk (32 rows x 128 columns) and a V chunk (32 rows x 32 columns) land in
//           the K-major 128-byte-swizzled layout the MMA reads (the column-major factor
//           is already K-major for both).  Six warps split a landed chunk into hi (in
//           place) and lo (one of 2 lo slots), one thread issues the 12 MMAs of the
//           chunk and frees both slots by commits, one thread refills landing slots.  The last CTA of
//           each column tile forms Z = T^T Y and writes it as the update's operand
//           image (Z^T hi and lo, swizzled).
//   k_vimg: V of the panel written once as the update's operand image (hi/lo, swizzled).
//   k_tcu : C -= V Z on 128 x 64 tiles (M = 128 rows, N = 64 columns, K = 32; two CTAs
//           per SM): the C tile arrives by TMA, the V image of its row block and its half
//           of the Z image by bulk copies; the epilogue subtracts D (tcgen05.ld) from the
//           staged C and stores coalesced along the rows.
// Every mbarrier wait is bounded: on timeout the kernel raises the device flag, waits
// (bounded) for its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "qr.cuh"
#include "tc_common.cuh"
#include "trail_z.cuh"

namespace {

constexpr int TY_C = 128;          // columns of C per k_tcy CTA (MMA M)
constexpr int TY_K = 32;           // rows per chunk (MMA K per stage)
constexpr int TY_THREADS = 256;
constexpr int TU_R = 128;          // rows per k_tcu tile (MMA M)
constexpr int TU_C = 64;           // columns per k_tcu tile (MMA N; two tiles per Z image)
constexpr int TU_THREADS = 256;
constexpr long long TC_SPIN = 2000000000ll;   // SM cycles (about a second) before a wait gives up

constexpr uint32_t TY_A = TY_C * 128;            // one 128 x 32 fp32 operand tile (bytes)
constexpr uint32_t TY_B = 32 * 128;              // one 32 x 32 fp32 operand tile
constexpr uint32_t TU_CT = TU_R * TU_C * 4;      // staged C tile
constexpr uint32_t TU_V = TU_R * 128;            // V hi (or lo)
constexpr uint32_t TU_Z = TU_C * 128;            // Z^T hi (or lo)

__device__ __forceinline__ unsigned char *align1024(unsigned char *p)
{
    const uint32_t a = tc::smem_addr(p);
    return p + ((1024u - (a & 1023u)) & 1023u);
}

__device__ __forceinline__ void expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

// 2-D tile of the factor (x = row, y = column) into shared memory, counted on bar
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3}], [%4];\n"
                 :: "r"(tc::smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
                    "r"(tc::smem_addr(bar))
                 : "memory");
}

// contiguous global -> shared copy (16-byte aligned, multiple of 16 bytes)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(tc::smem_addr(dst)), "l"(src), "r"(bytes), "r"(tc::smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(tc::smem_addr(bar)) : "memory");
}

__device__ __forceinline__ float v_at(const float *__restrict__ F, int64_t ld, int64_t k, int64_t i, int l,
                                      int ncols)
{
    if (l >= ncols || i < l) return 0.f;
    if (i == l) return 1.f;
    return F[(k + i) + (k + l) * ld];
}

__device__ __forceinline__ float4 split4(float4 &x)
{
    float4 lo;
    tc::split_tf32(x.x, x.x, lo.x);
    tc::split_tf32(x.y, x.y, lo.y);
    tc::split_tf32(x.z, x.z, lo.z);
    tc::split_tf32(x.w, x.w, lo.w);
    return lo;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// V of the panel at column k as the update's A operand: per block of 128 rows, the hi
// part then the lo part, each 128 rows x 32 fp32 in the K-major 128-byte-swizzled
// layout (thread = row, whole 128-byte rows written)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TU_R)
k_vimg(const float *__restrict__ F, int64_t ld, int64_t k, int ncols, int64_t mp, float *__restrict__ Vimg)
{
    const int r = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * TU_R + r;
    float x[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) x[l] = (i < mp) ? v_at(F, ld, k, i, l, ncols) : 0.f;
    float4 *hi = reinterpret_cast<float4 *>(Vimg + (int64_t)blockIdx.x * (2 * TU_R * 32) + r * 32);
    float4 *lo = hi + TU_R * 8;
#pragma unroll
    for (int c4 = 0; c4 < 8; ++c4) {
        float4 h = make_float4(x[4 * c4], x[4 * c4 + 1], x[4 * c4 + 2], x[4 * c4 + 3]);
        const float4 l4 = split4(h);
        const int phys = c4 ^ (r & 7);
        hi[phys] = h;
        lo[phys] = l4;
    }
}

// ---------------------------------------------------------------------------
// Y partials: Ypart[split][l][c] = sum over the split's rows of V(i, l) C(i, c).
// Warp roles: warp 0 loads chunks by TMA into a ring of TY_LAND landing slots, warps
// 2..7 split a landed chunk into hi (in place) and lo (into one of TY_LO lo slots),
// warp 1 issues the MMAs and commits them twice (freeing the landing slot and the lo
// slot).  Per-slot barriers: full (TMA landed), conv (split done), land_empty and
// lo_empty (MMAs done); no CTA-wide synchronisation inside the loop.
// ---------------------------------------------------------------------------
constexpr int TY_CONV = TY_THREADS / 32 - 2;     // converter warps
// Three landing slots and two lo slots: 100 KB of shared memory, so two CTAs (of one
// solve or of two solves on other streams) fit on an SM.  One solve at a time, 4 and 6
// landing slots ran at the same speed; with eight solves in flight, 3 slots gave 296
// solves/s against 272 with 4 or 6 (one CTA per SM).
constexpr int TY_LAND = 3;                       // landing slots (raw, then hi)
constexpr int TY_LO = 2;                         // lo slots
// Independent TMEM accumulators: the three split products of a chunk (hi*hi, hi*lo,
// lo*hi) and the chunk's parity each go to their own 32-column accumulator, so that
// consecutive MMAs do not wait on one accumulator; the epilogue adds the six.
constexpr int TY_NACC = 6;
constexpr uint32_t TY_TMEM = 256;                // columns allocated (power of two >= 6 x 32)
constexpr uint32_t TY_SLOT = TY_A + TY_B;        // one chunk: C part then V part
constexpr int TY_QA = TY_A / 16, TY_QB = TY_B / 16;                  // float4 per part
constexpr int TY_PER = (TY_QA + TY_QB + 32 * TY_CONV - 1) / (32 * TY_CONV);   // per converter thread

__global__ void __launch_bounds__(TY_THREADS, 1)
k_tcy(const __grid_constant__ CUtensorMap mC, const __grid_constant__ CUtensorMap mV, int64_t k, int ncols,
      int64_t nct, int64_t coff, int64_t mp, float *__restrict__ Ypart,
      float *__restrict__ Zimg, const float *__restrict__ Tblk, int *__restrict__ counters, int *flag)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = align1024(smem_raw);
    unsigned char *land = base, *lo = base + TY_LAND * TY_SLOT;
    __shared__ uint64_t full[TY_LAND], land_empty[TY_LAND], conv[TY_LO], lo_empty[TY_LO];
    __shared__ int s_last_load[TY_LAND], s_last_commit;
    __shared__ volatile int s_fail;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t cbase = (int64_t)blockIdx.x * TY_C;
    // chunk ch of this CTA is the panel's 32-row chunk blockIdx.y + ch * gridDim.y: the
    // CTAs of a column tile read neighbouring pieces of each column at the same time
    const int64_t tchunks = fl_cdiv_dev(mp, TY_K), S = gridDim.y;
    const int nchunks = (int)fl_max64(0, fl_cdiv_dev(tchunks - blockIdx.y, S));
    auto row0 = [&](int ch) { return ((int64_t)blockIdx.y + (int64_t)ch * S) * TY_K; };

    if (warp == 0) tc::tmem_alloc(&tmem_slot, TY_TMEM);
    if (threadIdx.x == 0) {
        for (int s = 0; s < TY_LAND; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&land_empty[s], 1);
            s_last_load[s] = -1;
        }
        for (int t = 0; t < TY_LO; ++t) {
            tc::mbar_init(&conv[t], TY_CONV);
            tc::mbar_init(&lo_empty[t], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_last_commit = -1;
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // TMA coordinates: x = row of the factor, y = column
            const int yc = (int)(k + ncols + coff + cbase), yv = (int)k;
            for (int ch = 0; ch < nchunks; ++ch) {
                const int s = ch % TY_LAND;
                if (ch >= TY_LAND &&
                    !tc::mbar_wait(&land_empty[s], (uint32_t)((ch - TY_LAND) / TY_LAND) & 1u, TC_SPIN)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                unsigned char *A = land + s * TY_SLOT;
                expect_tx(&full[s], TY_SLOT);
                tma_load_2d(A, &mC, (int)(k + row0(ch)), yc, &full[s]);
                tma_load_2d(A + TY_A, &mV, (int)(k + row0(ch)), yv, &full[s]);
                s_last_load[s] = ch;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_tf32(TY_C, 32);
            for (int ch = 0; ch < nchunks; ++ch) {
                const int s = ch % TY_LAND, t = ch % TY_LO;
                if (!tc::mbar_wait(&conv[t], (uint32_t)(ch / TY_LO) & 1u, TC_SPIN)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                tc::fence_after_sync();
                unsigned char *Ah = land + s * TY_SLOT, *Bh = Ah + TY_A, *Al = lo + t * TY_SLOT, *Bl = Al + TY_A;
                const uint64_t dAh = tc::smem_desc_sw128(Ah), dAl = tc::smem_desc_sw128(Al);
                const uint64_t dBh = tc::smem_desc_sw128(Bh), dBl = tc::smem_desc_sw128(Bl);
                // accumulators (parity of ch) x (hi*hi, hi*lo, lo*hi) at TMEM columns 32 a
                const uint32_t d0 = tmem + (uint32_t)(96 * (ch & 1));
#pragma unroll
                for (int ks = 0; ks < TY_K / 8; ++ks) {
                    const uint64_t o = (uint64_t)(ks * 32) >> 4;      // 8 tf32 = 32 bytes along K
                    const uint32_t acc = (ch > 1 || ks > 0) ? 1u : 0u;
                    tc::mma_tf32(d0, dAh + o, dBh + o, idesc, acc);
                    tc::mma_tf32(d0 + 32, dAh + o, dBl + o, idesc, acc);
                    tc::mma_tf32(d0 + 64, dAl + o, dBh + o, idesc, acc);
                }
                tc::mma_commit(&land_empty[s]);
                tc::mma_commit(&lo_empty[t]);
                s_last_commit = ch;
            }
            // the last commit arrives after every earlier MMA of the thread has completed
            if (!s_fail && nchunks > 0) {
                const int lc = nchunks - 1;
                if (!tc::mbar_wait(&lo_empty[lc % TY_LO], (uint32_t)(lc / TY_LO) & 1u, TC_SPIN)) s_fail = 1;
            }
        }
    } else {
        const int ct = threadIdx.x - 64;                 // 0 .. 32 TY_CONV - 1
        for (int ch = 0; ch < nchunks; ++ch) {
            const int s = ch % TY_LAND, t = ch % TY_LO;
            // the lo slot is free once the MMAs of chunk ch - TY_LO have completed
            if (ch >= TY_LO &&
                !tc::mbar_wait(&lo_empty[t], (uint32_t)((ch - TY_LO) / TY_LO) & 1u, TC_SPIN)) {
                s_fail = 1;
                break;
            }
            if (!tc::mbar_wait(&full[s], (uint32_t)(ch / TY_LAND) & 1u, TC_SPIN)) {
                s_fail = 1;
                break;
            }
            if (s_fail) break;
            float4 *hi = reinterpret_cast<float4 *>(land + s * TY_SLOT);
            float4 *lq = reinterpret_cast<float4 *>(lo + t * TY_SLOT);
            // float4 q < TY_QA: the C part; q >= TY_QA: the V part (smem row l = column l
            // of V, 4 consecutive rows) with zero past the panel's columns and the unit
            // lower triangle on the panel's top rows
            float4 x[TY_PER];
#pragma unroll
            for (int u = 0; u < TY_PER; ++u) {
                const int q = ct + u * 32 * TY_CONV;
                x[u] = (q < TY_QA + TY_QB) ? hi[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const int64_t r0 = row0(ch);
#pragma unroll
            for (int u = 0; u < TY_PER; ++u) {
                const int q = ct + u * 32 * TY_CONV;
                if (q >= TY_QA + TY_QB) continue;
                if (q >= TY_QA) {
                    const int qb = q - TY_QA, l = qb >> 3;
                    const int64_t i0 = r0 + (((qb & 7) ^ (l & 7)) << 2);
                    if (l >= ncols) {
                        x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else if (i0 <= l) {
                        x[u].x = (i0 + 0 < l) ? 0.f : ((i0 + 0 == l) ? 1.f : x[u].x);
                        x[u].y = (i0 + 1 < l) ? 0.f : ((i0 + 1 == l) ? 1.f : x[u].y);
                        x[u].z = (i0 + 2 < l) ? 0.f : ((i0 + 2 == l) ? 1.f : x[u].z);
                        x[u].w = (i0 + 3 < l) ? 0.f : ((i0 + 3 == l) ? 1.f : x[u].w);
                    }
                }
                const float4 l4 = split4(x[u]);
                hi[q] = x[u];
                lq[q] = l4;
            }
            tc::fence_proxy_async_smem();                // generic writes -> the MMA's reads
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[t]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool ok = !s_fail;
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
            // let the copies and MMAs in flight finish before the CTA leaves (bounded)
            for (int s = 0; s < TY_LAND; ++s)
                if (s_last_load[s] >= 0)
                    tc::mbar_wait(&full[s], (uint32_t)(s_last_load[s] / TY_LAND) & 1u, TC_SPIN);
            const int lc = s_last_commit;
            if (lc >= 0) tc::mbar_wait(&lo_empty[lc % TY_LO], (uint32_t)(lc / TY_LO) & 1u, TC_SPIN);
        }
    } else {
        // D: TMEM lane = column c, TMEM column = l; warp w reads lanes 32 (w % 4) ..
        // (its lane quarter) and columns 16 (w / 4) .. + 15
        const int q4 = warp & 3, lc = 16 * (warp >> 2);
        const int64_t c = cbase + q4 * 32 + lane;
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
        // the accumulators written: all six once there are two chunks, three with one
        const int nacc = nchunks > 1 ? TY_NACC : (nchunks > 0 ? 3 : 0);
        for (int a = 0; a < nacc; ++a) {
            float w[16];
            tc::tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(32 * a + lc), w);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] += w[j];
        }
        if (c < nct)
#pragma unroll
            for (int j = 0; j < 16; ++j) Ypart[((int64_t)blockIdx.y * 32 + lc + j) * nct + c] = v[j];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TY_TMEM);
    if (ok)   // uniform; the ring is free once the last MMA has completed
        trail_finish_z<float, 32, TY_C, TY_THREADS, true>(Ypart, (int)gridDim.y, nct, cbase, Tblk, Zimg,
                                                          counters + (int64_t)blockIdx.x * TREE_STRIDE,
                                                          counters + (int64_t)blockIdx.x * TREE_STRIDE + 1,
                                                          reinterpret_cast<float *>(base));
}

// ---------------------------------------------------------------------------
// C(i, c) -= sum_l V(i, l) Z(l, c) on a 128 x 64 tile
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TU_THREADS, 2)
k_tcu(const __grid_constant__ CUtensorMap mT, float *__restrict__ F, int64_t ld, int64_t k, int ncols,
      int64_t nct, int64_t coff, int64_t mp, const float *__restrict__ Vimg, const float *__restrict__ Zimg,
      int *flag)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = align1024(smem_raw);
    unsigned char *Vh = base, *Vl = Vh + TU_V, *Zh = Vl + TU_V, *Zl = Zh + TU_Z;
    const float *Cs = reinterpret_cast<const float *>(Zl + TU_Z);   // [c][r], r contiguous
    __shared__ uint64_t bar_c, bar_z, bar_m;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t rbase = (int64_t)blockIdx.x * TU_R;
    const int64_t cbase = (int64_t)blockIdx.y * TU_C;

    // three accumulators (hi*hi, hi*lo, lo*hi) of TU_C columns each, added in the epilogue,
    // so that consecutive MMAs do not wait on one accumulator; two CTAs per SM use 512
    if (warp == 0) tc::tmem_alloc(&tmem_slot, 4 * TU_C);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar_c, 1);
        tc::mbar_init(&bar_z, 1);
        tc::mbar_init(&bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        // the C tile (rows k + rbase .., columns of the update), the V image of the row
        // block and this tile's half of the Z image of its 128-column tile
        expect_tx(&bar_c, TU_CT);
        tma_load_2d(const_cast<float *>(Cs), &mT, (int)(k + rbase), (int)(k + ncols + coff + cbase), &bar_c);
        const float *img = Zimg + (cbase / TY_C) * (2 * TY_C * 32) + (cbase % TY_C) * 32;
        expect_tx(&bar_z, 2 * TU_V + 2 * TU_Z);
        bulk_load(Vh, Vimg + (int64_t)blockIdx.x * (2 * TU_R * 32), 2 * TU_V, &bar_z);   // hi, lo
        bulk_load(Zh, img, TU_Z, &bar_z);
        bulk_load(Zl, img + TY_C * 32, TU_Z, &bar_z);
    }
    const bool wz = tc::mbar_wait(&bar_z, 0u, TC_SPIN);
    tc::fence_before_sync();
    bool ok = __syncthreads_and(wz) != 0;
    tc::fence_after_sync();
    if (ok && threadIdx.x == 0) {
        constexpr uint32_t idesc = tc::idesc_tf32(TU_R, TU_C);
        const uint64_t dAh = tc::smem_desc_sw128(Vh), dAl = tc::smem_desc_sw128(Vl);
        const uint64_t dBh = tc::smem_desc_sw128(Zh), dBl = tc::smem_desc_sw128(Zl);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const uint64_t o = (uint64_t)(ks * 32) >> 4;
            const uint32_t acc = ks > 0 ? 1u : 0u;
            tc::mma_tf32(tmem, dAh + o, dBh + o, idesc, acc);
            tc::mma_tf32(tmem + TU_C, dAh + o, dBl + o, idesc, acc);
            tc::mma_tf32(tmem + 2 * TU_C, dAl + o, dBh + o, idesc, acc);
        }
        tc::mma_commit(&bar_m);
    }
    const bool wm = ok ? tc::mbar_wait(&bar_m, 0u, TC_SPIN) : true;
    const bool wc = tc::mbar_wait(&bar_c, 0u, TC_SPIN);
    const bool issued = ok;
    tc::fence_before_sync();
    ok = __syncthreads_and(ok && wm && wc) != 0;
    tc::fence_after_sync();
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
            tc::mbar_wait(&bar_c, 0u, TC_SPIN);
            tc::mbar_wait(&bar_z, 0u, TC_SPIN);
            if (issued) tc::mbar_wait(&bar_m, 0u, TC_SPIN);
        }
    } else {
        // D: TMEM lane = row, column = c.  Warp w reads lanes 32 (w % 4) .. (its lane
        // quarter), columns 32 (w / 4) .. + 31; C - D stored along the rows
        const int q4 = warp & 3, c0 = 32 * (warp >> 2);
        const int r = q4 * 32 + lane;
        const int64_t i = rbase + r;
#pragma unroll
        for (int cc = c0; cc < c0 + 32; cc += 16) {
            float v[16], w1[16], w2[16];
            const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + cc;
            tc::tmem_ld16(ta, v);
            tc::tmem_ld16(ta + TU_C, w1);
            tc::tmem_ld16(ta + 2 * TU_C, w2);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] += w1[j] + w2[j];
            if (i < mp) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t c = cbase + cc + j;
                    if (c < nct) F[(k + i) + (k + ncols + coff + c) * ld] = Cs[(cc + j) * TU_R + r] - v[j];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 4 * TU_C);
}

}  // namespace

namespace {

// the driver's tensor-map encoder, looked up once
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}
}  // namespace

// The factor F (ld rows x ntot columns, column-major fp32) seen as a 2-D tensor
// (dimension 0 = rows): boxes of box_r rows x box_c columns; out-of-range elements
// read as zero.
bool fl_encode_f32_map(CUtensorMap *m, const float *F, int64_t ld, int64_t ntot, uint32_t box_r, uint32_t box_c,
                       bool swizzle128)
{
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ntot};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {box_r, box_c};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(F), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {

// the three maps of one factor, cached (a factorisation launches two updates per panel)
struct FactorMaps {
    const float *F = nullptr;
    int64_t ld = 0, ntot = 0;
    CUtensorMap c, v, t;
};

bool factor_maps(const float *F, int64_t ld, int64_t ntot, FactorMaps &out)
{
    static std::mutex mu;
    static FactorMaps cache[8];
    static int next = 0;
    std::lock_guard<std::mutex> lock(mu);
    for (const FactorMaps &e : cache)
        if (e.F == F && e.ld == ld && e.ntot == ntot) {
            out = e;
            return true;
        }
    FactorMaps e;
    e.F = F;
    e.ld = ld;
    e.ntot = ntot;
    if (!fl_encode_f32_map(&e.c, F, ld, ntot, TY_K, TY_C, true) || !fl_encode_f32_map(&e.v, F, ld, ntot, TY_K, 32, true) ||
        !fl_encode_f32_map(&e.t, F, ld, ntot, TU_R, TU_C, false))
        return false;
    cache[next] = e;
    next = (next + 1) % 8;
    out = e;
    return true;
}

}  // namespace

// 1 when the tensor-core path does not take the shape (the caller uses the SIMT update)
int fl_trailing_tc_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols, int nb,
                       int64_t nct, int64_t coff, int64_t ntot, const float *Tblk, int *counters)
{
    if (nct <= 0) return 0;
    if (nb != 32 || ld % 4 != 0 || k % 4 != 0 || (reinterpret_cast<uintptr_t>(F) & 15u) != 0) return 1;
    FactorMaps maps;
    if (!factor_maps(F, ld, ntot, maps)) return 1;
    const size_t smem_y = (TY_LAND + TY_LO) * TY_SLOT + 1024;
    const size_t smem_u = 2 * TU_V + 2 * TU_Z + TU_CT + 1024;
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_tcy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_y);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tcu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_u);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "tensor-core attributes");
        attr_once.done(ctx->device);
    }
    const int64_t mp = m_aug - k;
    const int64_t ctiles = fl_cdiv(nct, TY_C);
    // one wave of k_tcy CTAs (one per SM) beside the 16-SM cluster of the next panel,
    // each streaming at least 16 chunks of rows
    const int64_t free_sms = std::max<int64_t>(1, ctx->num_sms - 16);
    const int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>({free_sms / ctiles, fl_cdiv(mp, 16 * TY_K),
                                                                    (int64_t)TREE_MAX_SPLITS}));
    const int64_t rblocks = fl_cdiv(mp, TU_R);
    float *Vimg = (float *)fl_ws(ctx, FL_WS_VIMG, (size_t)rblocks * 2 * TU_R * 32 * sizeof(float));
    float *Ypart = (float *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(float) * nsplit * 32 * nct);
    // Z image: per 128-column tile, hi and lo parts of 128 rows x 32 fp32
    float *Zimg = (float *)fl_ws(ctx, FL_WS_ZBUF, (size_t)ctiles * 2 * TY_C * 32 * sizeof(float));
    if (!Ypart || !Zimg || !Vimg) return FASTLSQ_ERR_NOMEM;
    FL_PROF_N(ctx, FASTLSQ_K_TRAIL_TC, 3);
    k_vimg<<<(unsigned)rblocks, TU_R, 0, ctx->stream>>>(F, ld, k, ncols, mp, Vimg);
    FL_CHECK_LAUNCH(ctx, "tc_vimg");
    k_tcy<<<dim3((unsigned)ctiles, (unsigned)nsplit), TY_THREADS, smem_y, ctx->stream>>>(
        maps.c, maps.v, k, ncols, nct, coff, mp, Ypart, Zimg, Tblk, counters, ctx->d_flag);
    FL_CHECK_LAUNCH(ctx, "tc_y");
    k_tcu<<<dim3((unsigned)rblocks, (unsigned)fl_cdiv(nct, TU_C)), TU_THREADS, smem_u, ctx->stream>>>(
        maps.t, F, ld, k, ncols, nct, coff, mp, Vimg, Zimg, ctx->d_flag);
    FL_CHECK_LAUNCH(ctx, "tc_update");
    return 0;
}

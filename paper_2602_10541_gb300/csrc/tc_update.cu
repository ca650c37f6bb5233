// Trailing update of the blocked Householder QR on the tcgen05 tensor cores, in
// split TF32x3 precision with FP32 accumulation in TMEM:
//   x = hi + lo (hi = tf32 rounding of x, lo = x - hi), a*b ~ ah*bh + ah*bl + al*bh.
// For panel k with Householder block V (m_p x nb, unit lower trapezoidal) and
// compact-WY factor T:
//   k_tc_y      : Y^T = C^T V over a split of the rows (M = 128 columns of C,
//                 N = nb, K = rows in chunks of 32), partial sums per split;
//   k_tc_update : C -= V Z with Z = T^T sum_s Y_s (M = 128 rows, N = 128 columns,
//                 K = nb).
// Operands are staged into shared memory by the warps (coalesced 128-byte loads),
// split into hi/lo and written in the K-major 128-byte-swizzle layout; one thread
// issues the MMAs and commits them to an mbarrier; the epilogue reads TMEM with
// tcgen05.ld.  Every mbarrier wait is bounded: on timeout the kernel raises the
// device flag, waits once more (bounded) and frees its TMEM.
#include <algorithm>

#include "common.cuh"
#include "qr.cuh"
#include "tc_common.cuh"
#include "trail_z.cuh"

namespace {

constexpr int TCY_COLS = 128;      // columns of C per CTA (M of the MMA)
constexpr int TCY_CHUNK = 32;      // rows per K-chunk
constexpr int TCU_ROWS = 128;      // rows of C per CTA in the update (M)
constexpr int TCU_COLS = 128;      // columns of C per CTA in the update (N)
constexpr long long TC_SPIN = 2000000000ll;   // SM cycles (about a second) before an mbarrier wait gives up

__device__ __forceinline__ float v_at_f(const float *__restrict__ F, int64_t ld, int64_t k, int64_t i,
                                        int l, int ncols)
{
    if (l >= ncols || i < l) return 0.f;
    if (i == l) return 1.f;
    return F[(k + i) + (k + l) * ld];
}

__device__ __forceinline__ unsigned char *align1024(unsigned char *p)
{
    const uint32_t a = tc::smem_addr(p);
    return p + ((1024u - (a & 1023u)) & 1023u);
}

// ---------------------------------------------------------------------------
// Y partials: Ypart[split][l][c] = sum over the split's rows of V(i, l) C(i, c)
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(128, 1)
k_tc_y(const float *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols, int64_t nct, int64_t coff,
       int64_t rows_per_split, float *__restrict__ Ypart, float *__restrict__ Z,
       const float *__restrict__ Tblk, int *__restrict__ counters, int *flag)
{
    constexpr int N = NB < 16 ? 16 : NB;                 // MMA N (multiple of 16 for M = 128)
    constexpr uint32_t A_BYTES = TCY_COLS * 128;         // 128 rows x 32 fp32
    constexpr uint32_t B_BYTES = N * 128;
    constexpr uint32_t STAGE = 2 * A_BYTES + 2 * B_BYTES; // hi/lo of A and B
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = align1024(smem_raw);
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t mp = m - k;
    const int64_t cbase = (int64_t)blockIdx.x * TCY_COLS;
    const int64_t rs0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t rs1 = fl_min64(mp, rs0 + rows_per_split);
    const int nchunks = (int)fl_max64(0, fl_cdiv_dev(rs1 - rs0, TCY_CHUNK));

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 32);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    constexpr uint32_t idesc = tc::idesc_tf32(128, N);
    bool ok = true;
    uint32_t uses[2] = {0u, 0u};

    for (int ch = 0; ch < nchunks && ok; ++ch) {
        const int buf = ch & 1;
        unsigned char *Ah = base + buf * STAGE, *Al = Ah + A_BYTES, *Bh = Al + A_BYTES, *Bl = Bh + B_BYTES;
        if (ch >= 2) {   // the MMAs that read this buffer two chunks ago must be done
            const bool w = tc::mbar_wait(&bar[buf], (uses[buf] - 1) & 1, TC_SPIN);
            ok = __syncthreads_and(w) != 0;          // uniform decision for the whole CTA
            if (!ok) break;
            tc::fence_after_sync();
        }
        const int64_t r0 = rs0 + (int64_t)ch * TCY_CHUNK;
        const int64_t i = r0 + lane;
        const bool iv = i < rs1;
        // A = C^T: smem row = column c (32 per warp), k = row within the chunk
#pragma unroll 8
        for (int cl = 0; cl < 32; ++cl) {
            const int cr = warp * 32 + cl;
            const int64_t c = cbase + cr;
            const float x = (iv && c < nct) ? F[(k + i) + (k + ncols + coff + c) * ld] : 0.f;
            float h, lo;
            tc::split_tf32(x, h, lo);
            const uint32_t off = tc::sw128_offset(cr, lane);
            *reinterpret_cast<float *>(Ah + off) = h;
            *reinterpret_cast<float *>(Al + off) = lo;
        }
        // B = V: smem row = l, k = row within the chunk
        for (int l = warp; l < N; l += 4) {
            const float x = (iv && l < NB) ? v_at_f(F, ld, k, i, l, ncols) : 0.f;
            float h, lo;
            tc::split_tf32(x, h, lo);
            const uint32_t off = tc::sw128_offset(l, lane);
            *reinterpret_cast<float *>(Bh + off) = h;
            *reinterpret_cast<float *>(Bl + off) = lo;
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x == 0) {
            const uint64_t dAh = tc::smem_desc_sw128(Ah), dAl = tc::smem_desc_sw128(Al);
            const uint64_t dBh = tc::smem_desc_sw128(Bh), dBl = tc::smem_desc_sw128(Bl);
#pragma unroll
            for (int ks = 0; ks < TCY_CHUNK / 8; ++ks) {
                const uint64_t o = (uint64_t)(ks * 32) >> 4;      // 8 tf32 = 32 bytes along K
                tc::mma_tf32(tmem, dAh + o, dBh + o, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
                tc::mma_tf32(tmem, dAh + o, dBl + o, idesc, 1u);
                tc::mma_tf32(tmem, dAl + o, dBh + o, idesc, 1u);
            }
            tc::mma_commit(&bar[buf]);
        }
        uses[buf] += 1;
    }
    // wait for the last chunk's MMAs (its commit completes after all earlier ones)
    if (ok && nchunks > 0) {
        const int lb = (nchunks - 1) & 1;
        ok = tc::mbar_wait(&bar[lb], (uses[lb] - 1) & 1, TC_SPIN);
    }
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
        if (threadIdx.x == 0) atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        for (int b2 = 0; b2 < 2; ++b2)
            if (uses[b2]) tc::mbar_wait(&bar[b2], (uses[b2] - 1) & 1, TC_SPIN);
    }
    tc::fence_after_sync();
    if (ok) {
        // D: TMEM lane = column c (warp w holds lanes 32w..32w+31), TMEM column = l
        const int64_t c = cbase + warp * 32 + lane;
#pragma unroll
        for (int lc = 0; lc < N; lc += 16) {
            float v[16];
            if (nchunks > 0) tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + lc, v);
            else
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int l = lc + j;
                if (l < NB && c < nct) Ypart[((int64_t)blockIdx.y * NB + l) * nct + c] = v[j];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 32);
    if (ok)   // uniform; the stage buffers are free once the last MMA has completed
        trail_finish_z<float, NB, TCY_COLS, 128>(Ypart, (int)gridDim.y, nct, cbase, Tblk, Z,
                                                 counters + blockIdx.x, reinterpret_cast<float *>(base));
}

// ---------------------------------------------------------------------------
// C(i, c) -= sum_l V(i, l) Z(l, c), Z = T^T Y
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(128, 1)
k_tc_update(float *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols, int64_t nct, int64_t coff,
            const float *__restrict__ Z, int *flag)
{
    constexpr uint32_t A_BYTES = TCU_ROWS * 128;     // 128 rows x 32 fp32 (K = l, padded to 32)
    constexpr uint32_t B_BYTES = TCU_COLS * 128;     // 128 columns x 32 fp32
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = align1024(smem_raw);
    unsigned char *Ah = base, *Al = Ah + A_BYTES, *Bh = Al + A_BYTES, *Bl = Bh + B_BYTES;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t mp = m - k;
    const int64_t rbase = (int64_t)blockIdx.x * TCU_ROWS;
    const int64_t cbase = (int64_t)blockIdx.y * TCU_COLS;

    if (warp == 0) tc::tmem_alloc(&tmem_slot, TCU_COLS);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // B = Z: thread t owns column c = cbase + t; smem row t, k = l
    {
        const int64_t c = cbase + threadIdx.x;
        float zl[NB];
#pragma unroll
        for (int l = 0; l < NB; ++l) zl[l] = (c < nct) ? Z[(int64_t)l * nct + c] : 0.f;
#pragma unroll
        for (int l = 0; l < 32; ++l) {
            const float z = (l < NB) ? zl[l] : 0.f;
            float h, lo;
            tc::split_tf32(z, h, lo);
            const uint32_t off = tc::sw128_offset(threadIdx.x, l);
            *reinterpret_cast<float *>(Bh + off) = h;
            *reinterpret_cast<float *>(Bl + off) = lo;
        }
    }
    // A = V rows: warp w stages rows 32w..32w+31, lane = row, loop over l (coalesced)
    {
        const int r = warp * 32 + lane;
        const int64_t i = rbase + r;
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
            const float x = (i < mp && l < NB) ? v_at_f(F, ld, k, i, l, ncols) : 0.f;
            float h, lo;
            tc::split_tf32(x, h, lo);
            const uint32_t off = tc::sw128_offset(r, l);
            *reinterpret_cast<float *>(Ah + off) = h;
            *reinterpret_cast<float *>(Al + off) = lo;
        }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        constexpr uint32_t idesc = tc::idesc_tf32(TCU_ROWS, TCU_COLS);
        const uint64_t dAh = tc::smem_desc_sw128(Ah), dAl = tc::smem_desc_sw128(Al);
        const uint64_t dBh = tc::smem_desc_sw128(Bh), dBl = tc::smem_desc_sw128(Bl);
#pragma unroll
        for (int ks = 0; ks < (NB + 7) / 8; ++ks) {
            const uint64_t o = (uint64_t)(ks * 32) >> 4;
            tc::mma_tf32(tmem, dAh + o, dBh + o, idesc, ks > 0 ? 1u : 0u);
            tc::mma_tf32(tmem, dAh + o, dBl + o, idesc, 1u);
            tc::mma_tf32(tmem, dAl + o, dBh + o, idesc, 1u);
        }
        tc::mma_commit(&bar);
    }
    bool ok = __syncthreads_and(tc::mbar_wait(&bar, 0, TC_SPIN)) != 0;
    if (!ok) {
        if (threadIdx.x == 0) atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        tc::mbar_wait(&bar, 0, TC_SPIN);
    }
    tc::fence_after_sync();
    if (ok) {
        // D: TMEM lane = row (warp w: rows 32w..), column = c; C -= D, coalesced along rows
        const int64_t i = rbase + warp * 32 + lane;
#pragma unroll 1
        for (int cc = 0; cc < TCU_COLS; cc += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cc, v);
            if (i < mp) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t c = cbase + cc + j;
                    if (c < nct) {
                        float *p = F + (k + i) + (k + ncols + coff + c) * ld;
                        *p -= v[j];
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TCU_COLS);
}

template <int NB>
int launch_tc(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols, int64_t nct,
              int64_t coff, const float *Tblk, int *counters)
{
    constexpr int N = NB < 16 ? 16 : NB;
    const size_t smem_y = 2 * (2 * TCY_COLS * 128 + 2 * N * 128) + 1024;
    const size_t smem_u = 2 * TCU_ROWS * 128 + 2 * TCU_COLS * 128 + 1024;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_y<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_y);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_tc_update<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_u);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "tensor-core attributes");
        attr_done = true;
    }
    const int64_t mp = m_aug - k;
    const int64_t ctiles = fl_cdiv(nct, TCY_COLS);
    int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>(fl_cdiv(2 * ctx->num_sms, ctiles), fl_cdiv(mp, 256)));
    int64_t rows_per_split = fl_round_up(fl_cdiv(mp, nsplit), TCY_CHUNK);
    nsplit = fl_cdiv(mp, rows_per_split);
    float *Ypart = (float *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(float) * nsplit * NB * nct);
    float *Z = (float *)fl_ws(ctx, FL_WS_ZBUF, sizeof(float) * NB * nct);
    if (!Ypart || !Z) return FASTLSQ_ERR_NOMEM;
    FL_PROF_N(ctx, FASTLSQ_K_TRAIL_TC, 2);
    k_tc_y<NB><<<dim3((unsigned)ctiles, (unsigned)nsplit), 128, smem_y, ctx->stream>>>(
        F, ld, k, m_aug, ncols, nct, coff, rows_per_split, Ypart, Z, Tblk, counters, ctx->d_flag);
    FL_CHECK_LAUNCH(ctx, "tc_y");
    k_tc_update<NB><<<dim3((unsigned)fl_cdiv(mp, TCU_ROWS), (unsigned)fl_cdiv(nct, TCU_COLS)), 128, smem_u,
                      ctx->stream>>>(F, ld, k, m_aug, ncols, nct, coff, Z, ctx->d_flag);
    FL_CHECK_LAUNCH(ctx, "tc_update");
    return 0;
}

}  // namespace

int fl_trailing_tc_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                       int nb, int64_t nct, int64_t coff, const float *Tblk, int *counters)
{
    if (nct <= 0) return 0;
    switch (nb) {
    case 32: return launch_tc<32>(ctx, F, ld, k, m_aug, ncols, nct, coff, Tblk, counters);
    case 16: return launch_tc<16>(ctx, F, ld, k, m_aug, ncols, nct, coff, Tblk, counters);
    case 8: return launch_tc<8>(ctx, F, ld, k, m_aug, ncols, nct, coff, Tblk, counters);
    default: return fl_fail(ctx, FASTLSQ_ERR_INVALID, "tensor-core update: panel width %d", nb);
    }
}

// Outer-block trailing update of the two-level blocked Householder QR on the tcgen05
// tensor cores (Sec. 2.3 "via QR"), in a three-part bf16 split with FP32 accumulation:
//
//   x = x1 + x2 + x3,  x1 = bf16(x), x2 = bf16(x - x1), x3 = x - x1 - x2 (exact in bf16
//   for every normal fp32 x: 8 + 8 + 8 significand bits cover fp32's 24), and
//   a*b ~ a1 b1 + (a1 b2 + a2 b1 + a1 b3 + a3 b1 + a2 b2);
//
// the dropped terms (a2 b3, a3 b2, a3 b3) are below 2^-25 |ab|, so the products carry
// FP32-level accuracy (the TF32x3 split of the per-panel update carries 2^-22).  The
// tensor core sums at most 64 rows (the Y pass) or 64 block columns (the update pass,
// with the leading product a1 b1 and the five small ones in separate accumulators)
// before the sums continue in FP32 registers with round-to-nearest adds.  Six bf16
// products cost what three tf32 ones do (bf16 runs at twice the tf32 rate).
//
// For an outer block of nbk <= 128 columns at column k, already factored as inner
// panels of width NB (their reflectors V in F below the diagonal, their NB x NB
// compact-WY factors T_q in the factor's T storage), the trailing columns C (the rest
// of F, right-hand sides included) get C <- H^T C, H = H_0 H_1 ... H_{nq-1}:
//   k_bimg : V of the block written once as two bf16 operand images (three parts
//            each, K-major, 128-byte swizzle): VY (rows of V^T, K = factor rows, per
//            64-row chunk) for the Y pass and VU (rows of V, K = block columns, per
//            128-row tile) for the update pass;
//   k_by   : Y = V^T [V | C] over split row ranges (MMA M = 128 block columns, N = 128
//            columns, K = 64 rows per stage); the columns of C are loaded from F by
//            converter warps (coalesced float4 along the rows), split in registers and
//            stored in the operand layout; the leading products of each 64-row chunk
//            accumulate in a fresh TMEM accumulator that the converter warps add into
//            FP32 registers two chunks behind the MMAs (the small products accumulate
//            over the split in TMEM); the V^T V
//            block (Gram matrix) comes out of the same pass from the block's own columns
//            (unit lower trapezoid applied); k_bsum adds the split partials in order;
//   k_bz   : Z = the block-triangular T^T applied to Y, inner panel by inner panel:
//            Z_q = T_q^T (Y_q - sum_{p<q} (V_p^T V_q)^T Z_p)  (the compact-WY product of
//            the inner panels), written as the update's bf16 operand image;
//   k_bu   : C -= V Z (M = 128 rows, N = 64 columns, K = 128), persistent CTAs over
//            (row tile, column tile) units with the VU tile resident, Z tiles in a ring
//            of two and two TMEM accumulator buffers, so the epilogue (C read, C - D
//            written, coalesced along the rows) overlaps the next tile's MMAs.
// Every mbarrier wait is bounded: on timeout the kernel raises the device flag, waits
// (bounded) for its copies and MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "qr.cuh"
#include "tc_common.cuh"

namespace {

constexpr int BK = 128;                 // outer block width (MMA M of the Y pass, K of the update)
constexpr int BY_KC = 64;               // factor rows per Y-pass stage (128 bytes of bf16)
constexpr int BY_N = 128;               // columns per Y-pass CTA
constexpr int BU_R = 128;               // rows per update tile
constexpr int BU_N = 64;                // columns per update tile
constexpr uint32_t PART128 = 128u * 128u;         // one part of a 128-row operand tile (bytes)
constexpr uint32_t ZPART = BU_N * 128u;            // one part of a 64-row operand tile
constexpr uint32_t VY_CHUNK = 3u * PART128;        // VY image of one 64-row chunk
constexpr uint32_t VU_TILE = 6u * PART128;         // VU image of one 128-row tile (2 K halves)
constexpr uint32_t Z_TILE = 6u * ZPART;            // Z image of one 64-column tile
constexpr long long BT_SPIN = 2000000000ll;        // SM cycles (about a second) before a wait gives up

// 10 warps: three share an SM sub-partition's 16K registers, so at most 168 a thread
constexpr int BY_THREADS = 320;         // warp 0: A loads, warp 1: MMA, warps 2..9: converters, epilogue
constexpr int BY_CONV = 8;
constexpr uint32_t BY_STAGE = 2u * VY_CHUNK;       // A parts then B parts
constexpr uint32_t BY_RAW = 64u * BY_N * 4u;       // one chunk of F as fp32 (64 rows x 128 columns)
constexpr size_t BY_SMEM = 2 * BY_STAGE + BY_RAW + 1024;
constexpr int BY_PF = 3;                // chunks ahead that the converters prefetch into L2
constexpr int BU_THREADS = 320;         // warp 0: loads, warp 1: MMA, warps 2..9: epilogue
constexpr int BU_EPI = 8;
constexpr uint32_t BU_CT = (uint32_t)BU_R * BU_N * 4u;   // one tile of C as fp32 (128 rows x 64 columns)
constexpr size_t BU_SMEM = VU_TILE + 2 * Z_TILE + BU_CT + 1024;
constexpr int BI_LD = 129;              // padded row of the k_bimg staging tile
constexpr size_t BI_SMEM = sizeof(float) * 128 * BI_LD;

__device__ __forceinline__ unsigned char *bt_align1024(unsigned char *p)
{
    const uint32_t a = tc::smem_addr(p);
    return p + ((1024u - (a & 1023u)) & 1023u);
}

__device__ __forceinline__ void bt_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bt_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(tc::smem_addr(dst)), "l"(src), "r"(bytes), "r"(tc::smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void bt_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" :: "r"(tc::smem_addr(bar)) : "memory");
}

// 2-D tile of F (x = row, y = column) into shared memory, counted on bar; rows and
// columns outside F read as zero
__device__ __forceinline__ void bt_tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                 "[%0], [%1, {%2, %3}], [%4];\n"
                 :: "r"(tc::smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y),
                    "r"(tc::smem_addr(bar))
                 : "memory");
}

// Operand tiles are K-major with 128-byte rows (64 bf16 along K) in the 128-byte
// swizzle: element (row, kk) sits at row * 128 + (((kk / 8) ^ (row % 8)) * 16) + 2 (kk % 8).
// three-part split of two fp32 values with paired conversions (one cvt per pair and part)
__device__ __forceinline__ void split3x2(float x, float y, uint32_t &a, uint32_t &b, uint32_t &c)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);              // .x = x (low half)
    const float rx = x - __low2float(h), ry = y - __high2float(h);
    const __nv_bfloat162 m = __floats2bfloat162_rn(rx, ry);
    const __nv_bfloat162 l = __floats2bfloat162_rn(rx - __low2float(m), ry - __high2float(m));
    a = *reinterpret_cast<const uint32_t *>(&h);
    b = *reinterpret_cast<const uint32_t *>(&m);
    c = *reinterpret_cast<const uint32_t *>(&l);
}

// 4 consecutive K elements -> three parts of 8 bytes each
__device__ __forceinline__ void split4(float4 v, uint2 (&p)[3])
{
    split3x2(v.x, v.y, p[0].x, p[1].x, p[2].x);
    split3x2(v.z, v.w, p[0].y, p[1].y, p[2].y);
}

// 8 consecutive K elements -> three parts of 16 bytes each
__device__ __forceinline__ void split8(const float (&v)[8], uint4 (&p)[3])
{
    split3x2(v[0], v[1], p[0].x, p[1].x, p[2].x);
    split3x2(v[2], v[3], p[0].y, p[1].y, p[2].y);
    split3x2(v[4], v[5], p[0].z, p[1].z, p[2].z);
    split3x2(v[6], v[7], p[0].w, p[1].w, p[2].w);
}

// V(i, l) of the block: unit lower trapezoid, zero past the block's nbk columns
__device__ __forceinline__ float v_mask(float raw, int64_t i, int l, int nbk)
{
    if (l >= nbk || i < l) return 0.f;
    return (i == l) ? 1.f : raw;
}

// ---------------------------------------------------------------------------
// k_bimg: one CTA per 128-row tile t of the block's rows (panel-local rows
// 128 t .. 128 t + 127).  The tile of V (128 rows x 128 columns) is staged in shared
// memory, then written as the VU tile (row-major operand, K = block column) and as
// the VY chunks 2t and 2t + 1 (column-major operand, K = row).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_bimg(const float *__restrict__ F, int64_t ld, int64_t k, int nbk, int64_t mp, int64_t nch,
       unsigned char *__restrict__ VY, unsigned char *__restrict__ VU)
{
    extern __shared__ float sx[];          // sx[l * BI_LD + r]
    const int64_t t = blockIdx.x;
    const int tid = threadIdx.x;
    // the tile's 128 rows x 128 block columns: every load of a thread issued before its
    // stores, in two halves of eight (a loop of dependent load-store pairs left one memory
    // round trip per iteration exposed)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float4 v[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int idx = tid + (half * 8 + it) * 256, l = idx >> 5, q4 = idx & 31;
            const int64_t i = t * 128 + 4 * q4;             // panel-local row of the quad
            v[it] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l < nbk && i < mp && k + i < ld) v[it] = *reinterpret_cast<const float4 *>(F + (k + i) + (k + l) * ld);
        }
        asm volatile("" ::: "memory");                   // the loads above stay ahead of the stores
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int idx = tid + (half * 8 + it) * 256, l = idx >> 5, q4 = idx & 31;
            const int64_t i = t * 128 + 4 * q4;
            float *d = sx + l * BI_LD + 4 * q4;
            d[0] = (i + 0 < mp) ? v_mask(v[it].x, i + 0, l, nbk) : 0.f;
            d[1] = (i + 1 < mp) ? v_mask(v[it].y, i + 1, l, nbk) : 0.f;
            d[2] = (i + 2 < mp) ? v_mask(v[it].z, i + 2, l, nbk) : 0.f;
            d[3] = (i + 3 < mp) ? v_mask(v[it].w, i + 3, l, nbk) : 0.f;
        }
    }
    __syncthreads();
    // VU: row r, 16 chunks of 8 block columns (two K halves of 8 chunks)
    unsigned char *vu = VU + t * VU_TILE;
    for (int idx = tid; idx < 128 * 16; idx += 256) {
        const int r = idx >> 4, c16 = idx & 15, h = c16 >> 3, cc = c16 & 7;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = sx[(8 * c16 + e) * BI_LD + r];
        uint4 p[3];
        split8(v, p);
        const uint32_t off = (uint32_t)r * 128u + (((uint32_t)cc ^ ((uint32_t)r & 7u)) << 4);
#pragma unroll
        for (int q = 0; q < 3; ++q)
            *reinterpret_cast<uint4 *>(vu + (uint32_t)(h * 3 + q) * PART128 + off) = p[q];
    }
    // VY: chunks 2t, 2t + 1; row l of the chunk, 8 chunks of 8 factor rows
    for (int qq = 0; qq < 2; ++qq) {
        const int64_t q = 2 * t + qq;
        if (q >= nch) break;
        unsigned char *vy = VY + q * VY_CHUNK;
        for (int idx = tid; idx < 128 * 8; idx += 256) {
            const int l = idx >> 3, c8 = idx & 7;
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = sx[l * BI_LD + 64 * qq + 8 * c8 + e];
            uint4 p[3];
            split8(v, p);
            const uint32_t off = (uint32_t)l * 128u + (((uint32_t)c8 ^ ((uint32_t)l & 7u)) << 4);
#pragma unroll
            for (int pp = 0; pp < 3; ++pp) *reinterpret_cast<uint4 *>(vy + (uint32_t)pp * PART128 + off) = p[pp];
        }
    }
}
// ---------------------------------------------------------------------------
// k_by: Ypart[s][e][l] = sum over the split's rows i of V(i, l) X(i, e), X = F's
// columns k + e (e < nbk: the block's own V, masked; e >= nbk: the trailing columns).
// CTA (j, s): columns e in [128 j, 128 j + 128), the 64-row chunks s, s + S, ...
// Roles: warp 0 bulk-loads the VY chunk (A operand, three parts) (lane 0) and the raw
// fp32 X chunk of F by TMA into one raw buffer (lane 1) as soon as the converters have
// read the previous one, warps 2..9 read the X chunk into registers one chunk ahead
// (so a chunk of F is requested two chunks before its parts are stored; and three
// ahead into L2), split it and store the three B parts, warp 1 issues
// the 24 MMAs of the chunk, commits each 32-row half to that half's accumulator and the
// whole chunk to the stage's "empty" barrier.  The five small products accumulate over
// the whole split in one TMEM accumulator; each half-chunk's leading products go to a
// fresh TMEM accumulator (three buffers in turn) that warps 2..9 add into FP32
// registers one chunk behind the MMAs, so the long sum of the leading products over
// the split's rows is taken with round-to-nearest adds while the tensor core sums only
// 32 rows at a time, and the adds stay off the MMAs' path.  (Measured: sharing one accumulator between the leading and
// the small products, even for 64 rows, made R a worse CGLS preconditioner.)
// ---------------------------------------------------------------------------
constexpr int BY_NBUF = 3;             // leading-product accumulators in TMEM (plus the small one)

__global__ void __launch_bounds__(BY_THREADS, 1)
k_by(const __grid_constant__ CUtensorMap mF, const float *__restrict__ F, int64_t ld, int64_t k, int nbk,
     int64_t mp, int64_t n_ext, const unsigned char *__restrict__ VY, int64_t nch, float *__restrict__ Ypart,
     int *flag)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = bt_align1024(smem_raw);
    const float *raw = reinterpret_cast<const float *>(base + 2 * BY_STAGE);   // [128 columns][64 rows]
    __shared__ uint64_t fullA[2], fullB[2], empty[2], accf[BY_NBUF], acce[BY_NBUF], rawFull, rawEmpty;
    __shared__ int s_last_load[2], s_last_commit, s_last_raw;
    __shared__ volatile int s_fail;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ebase = (int64_t)blockIdx.x * BY_N;
    const int64_t S = gridDim.y;
    const int nloc = (int)fl_max64(0, fl_cdiv_dev(nch - (int64_t)blockIdx.y, S));
    auto chunk = [&](int ch) { return (int64_t)blockIdx.y + (int64_t)ch * S; };

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&fullA[s], 1);
            tc::mbar_init(&fullB[s], BY_CONV);
            tc::mbar_init(&empty[s], 1);
            s_last_load[s] = -1;
        }
        for (int b = 0; b < BY_NBUF; ++b) {
            tc::mbar_init(&accf[b], 1);
            tc::mbar_init(&acce[b], BY_CONV);
        }
        tc::mbar_init(&rawFull, 1);
        tc::mbar_init(&rawEmpty, BY_CONV);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_last_commit = -1;
        s_last_raw = -1;
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    // TMEM columns: [0, 128) the small products of the split, [128 + 128 b, 256 + 128 b)
    // the leading products of half-chunk buffer b
    const uint32_t tsmall = tmem;

    if (warp == 0) {
        if (lane == 0) {
            for (int ch = 0; ch < nloc; ++ch) {
                const int s = ch & 1;
                if (ch >= 2 && !tc::mbar_wait(&empty[s], (uint32_t)((ch - 2) >> 1) & 1u, BT_SPIN)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                bt_expect_tx(&fullA[s], VY_CHUNK);
                bt_bulk_load(base + s * BY_STAGE, VY + chunk(ch) * VY_CHUNK, VY_CHUNK, &fullA[s]);
                s_last_load[s] = ch;
            }
        } else if (lane == 1) {
            // the raw chunks of F by TMA into the one raw buffer, once the converters have
            // read the previous chunk out of it
            for (int ch = 0; ch < nloc; ++ch) {
                if (ch >= 1 && !tc::mbar_wait(&rawEmpty, (uint32_t)(ch - 1) & 1u, BT_SPIN)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                bt_expect_tx(&rawFull, BY_RAW);
                bt_tma_2d(base + 2 * BY_STAGE, &mF, (int)(k + chunk(ch) * BY_KC), (int)(k + ebase), &rawFull);
                s_last_raw = ch;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(BK, BY_N);
            for (int ch = 0; ch < nloc && !s_fail; ++ch) {
                const int s = ch & 1;
                if (!tc::mbar_wait(&fullA[s], (uint32_t)(ch >> 1) & 1u, BT_SPIN) ||
                    !tc::mbar_wait(&fullB[s], (uint32_t)(ch >> 1) & 1u, BT_SPIN)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                tc::fence_after_sync();
                const unsigned char *A = base + s * BY_STAGE, *B = A + VY_CHUNK;
                uint64_t dA[3], dB[3];
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    dA[p] = tc::smem_desc_sw128(A + p * PART128);
                    dB[p] = tc::smem_desc_sw128(B + p * PART128);
                }
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    // half-chunk hc: rows [32 hh, 32 hh + 32) of the chunk, its leading
                    // products into buffer hc mod 3 once the converters have drained it
                    const int hc = 2 * ch + hh, b = hc % BY_NBUF;
                    if (hc >= BY_NBUF &&
                        !tc::mbar_wait(&acce[b], (uint32_t)((hc - BY_NBUF) / BY_NBUF) & 1u, BT_SPIN)) {
                        s_fail = 1;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t dbig = tmem + (uint32_t)(BY_N + BY_N * b);
#pragma unroll
                    for (int kk = 0; kk < BY_KC / 32; ++kk) {
                        const int ks = (BY_KC / 32) * hh + kk;
                        const uint64_t o = (uint64_t)(ks * 32) >> 4;   // 16 bf16 = 32 bytes along K
                        tc::mma_bf16(dbig, dA[0] + o, dB[0] + o, idesc, kk > 0 ? 1u : 0u);
                        tc::mma_bf16(tsmall, dA[0] + o, dB[1] + o, idesc, (ch > 0 || ks > 0) ? 1u : 0u);
                        tc::mma_bf16(tsmall, dA[1] + o, dB[0] + o, idesc, 1u);
                        tc::mma_bf16(tsmall, dA[0] + o, dB[2] + o, idesc, 1u);
                        tc::mma_bf16(tsmall, dA[2] + o, dB[0] + o, idesc, 1u);
                        tc::mma_bf16(tsmall, dA[1] + o, dB[1] + o, idesc, 1u);
                    }
                    tc::mma_commit(&accf[b]);
                    s_last_commit = hc;
                }
                if (s_fail) break;
                tc::mma_commit(&empty[s]);
            }
        }
    } else {
        const int ct = threadIdx.x - 64;                       // 0 .. 255
        // D: TMEM lane = block column l, column = e.  Warp w adds its lane quarter
        // (w mod 4) and half (w - 2) / 4 of the 128 columns into its registers
        const int qd = warp & 3, hf = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
        float y[64];
#pragma unroll
        for (int jj = 0; jj < 64; ++jj) y[jj] = 0.f;
        float4 x[8];
        // chunk ch from the raw buffer (TMA-loaded; rows and columns outside F are zero)
        auto load = [&](int ch) -> bool {
            if (!tc::mbar_wait(&rawFull, (uint32_t)ch & 1u, BT_SPIN)) return false;
            const int64_t r0 = chunk(ch) * BY_KC;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = ct + 256 * u, cc = q >> 4, quad = q & 15;
                const int64_t i = r0 + 4 * quad;               // panel-local row
                const int64_t e = ebase + cc;
                float4 v = *reinterpret_cast<const float4 *>(raw + cc * BY_KC + 4 * quad);
                if (e < nbk) {
                    v.x = (i + 0 < mp) ? v_mask(v.x, i + 0, (int)e, nbk) : 0.f;
                    v.y = (i + 1 < mp) ? v_mask(v.y, i + 1, (int)e, nbk) : 0.f;
                    v.z = (i + 2 < mp) ? v_mask(v.z, i + 2, (int)e, nbk) : 0.f;
                    v.w = (i + 3 < mp) ? v_mask(v.w, i + 3, (int)e, nbk) : 0.f;
                }
                x[u] = v;
            }
            __syncwarp();
            if (lane == 0) bt_arrive(&rawEmpty);
            return true;
        };
        // y += leading products of half-chunk hc
        auto drain = [&](int hc) -> bool {
            const int b = hc % BY_NBUF;
            if (!tc::mbar_wait(&accf[b], (uint32_t)(hc / BY_NBUF) & 1u, BT_SPIN)) return false;
            tc::fence_after_sync();
#pragma unroll
            for (int rd = 0; rd < 2; ++rd) {
                uint32_t v0[16], v1[16];
                const uint32_t src = tmem + lane_base + (uint32_t)(BY_N + BY_N * b + 64 * hf + 32 * rd);
                tc::tmem_ld16_nw(src, v0);
                tc::tmem_ld16_nw(src + 16, v1);
                tc::tmem_wait_ld();
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    y[32 * rd + jj] += __uint_as_float(v0[jj]);
                    y[32 * rd + 16 + jj] += __uint_as_float(v1[jj]);
                }
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) bt_arrive(&acce[b]);
            return true;
        };
        if (nloc > 0 && !load(0)) s_fail = 1;
        for (int ch = 0; ch < nloc; ++ch) {
            const int s = ch & 1;
            if (ch >= 2 && !tc::mbar_wait(&empty[s], (uint32_t)((ch - 2) >> 1) & 1u, BT_SPIN)) {
                s_fail = 1;
                break;
            }
            if (s_fail) break;
            unsigned char *B = base + s * BY_STAGE + VY_CHUNK;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = ct + 256 * u, cc = q >> 4, quad = q & 15;
                uint2 p[3];
                split4(x[u], p);
                const uint32_t off = (uint32_t)cc * 128u + ((((uint32_t)quad >> 1) ^ ((uint32_t)cc & 7u)) << 4) +
                                     (((uint32_t)quad & 1u) << 3);
#pragma unroll
                for (int pp = 0; pp < 3; ++pp) *reinterpret_cast<uint2 *>(B + (uint32_t)pp * PART128 + off) = p[pp];
            }
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) bt_arrive(&fullB[s]);
            if (ch + 1 < nloc && !load(ch + 1)) {
                s_fail = 1;
                break;
            }
            if (ch + BY_PF < nloc) {   // the chunk BY_PF ahead into L2: thread (column ct / 2, half ct % 2)
                const int64_t ip = chunk(ch + BY_PF) * BY_KC + 32 * (ct & 1);
                const int64_t ep = ebase + (ct >> 1);
                if (ep < n_ext && ip < mp)
                    asm volatile("prefetch.global.L2 [%0];\n" :: "l"(F + (k + ip) + (k + ep) * ld));
            }
            if (ch >= 1 && (!drain(2 * ch - 2) || !drain(2 * ch - 1))) {
                s_fail = 1;
                break;
            }
        }
        if (nloc > 0 && !s_fail && (!drain(2 * nloc - 2) || !drain(2 * nloc - 1))) s_fail = 1;
        __syncwarp();
        if (!s_fail) {
            // the small products of the whole split (every MMA has completed: the last
            // chunk's commit arrived after all earlier MMAs of the issuing thread)
            const int l = 32 * qd + lane;
#pragma unroll
            for (int rd = 0; rd < 4; ++rd) {
                float t[16];
                const uint32_t col = (uint32_t)(64 * hf + 16 * rd);
                if (nloc > 0) tc::tmem_ld16(tsmall + lane_base + col, t);
                else
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) t[jj] = 0.f;
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) {
                    const int64_t e = ebase + col + jj;
                    if (e < n_ext) Ypart[((int64_t)blockIdx.y * n_ext + e) * BK + l] = y[16 * rd + jj] + t[jj];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (s_fail) {
        if (threadIdx.x == 0) {
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
            for (int s = 0; s < 2; ++s)
                if (s_last_load[s] >= 0) tc::mbar_wait(&fullA[s], (uint32_t)(s_last_load[s] >> 1) & 1u, BT_SPIN);
            const int lc = s_last_commit;
            if (lc >= 0) tc::mbar_wait(&accf[lc % BY_NBUF], (uint32_t)(lc / BY_NBUF) & 1u, BT_SPIN);
            if (s_last_raw >= 0) tc::mbar_wait(&rawFull, (uint32_t)s_last_raw & 1u, BT_SPIN);
        }
        __syncthreads();
    }
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// k_bsum: Ysum[e][l] = sum over the splits s (in split order) of Ypart[s][e][l]; one
// warp per column e, four block columns l per lane.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_bsum(const float *__restrict__ Ypart, int S, int64_t n_ext, float *__restrict__ Ysum)
{
    const int64_t e = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= n_ext) return;
    const float4 *src = reinterpret_cast<const float4 *>(Ypart + e * BK) + lane;
    const int64_t stride = n_ext * (BK / 4);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int s = 0;
    for (; s + 4 <= S; s += 4) {
        const float4 a0 = __ldcg(src + (int64_t)s * stride), a1 = __ldcg(src + (int64_t)(s + 1) * stride);
        const float4 a2 = __ldcg(src + (int64_t)(s + 2) * stride), a3 = __ldcg(src + (int64_t)(s + 3) * stride);
        acc.x = (((acc.x + a0.x) + a1.x) + a2.x) + a3.x;
        acc.y = (((acc.y + a0.y) + a1.y) + a2.y) + a3.y;
        acc.z = (((acc.z + a0.z) + a1.z) + a2.z) + a3.z;
        acc.w = (((acc.w + a0.w) + a1.w) + a2.w) + a3.w;
    }
    for (; s < S; ++s) {
        const float4 a = __ldcg(src + (int64_t)s * stride);
        acc.x += a.x;
        acc.y += a.y;
        acc.z += a.z;
        acc.w += a.w;
    }
    reinterpret_cast<float4 *>(Ysum + e * BK)[lane] = acc;
}

// ---------------------------------------------------------------------------
// k_bz: one CTA per 64 trailing columns.  Y (block columns x 64) and the Gram matrix
// G = V^T V come from Ysum; then, inner panel by inner panel, W_q = Y_q - sum_{p<q}
// (V_p^T V_q)^T Z_p and Z_q = T_q^T W_q; Z is written as the update's B-operand image
// (64 rows = columns, K = block column, three parts).
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(256)
k_bz(const float *__restrict__ Ysum, int64_t n_ext, int nbk, const float *__restrict__ Tb,
     unsigned char *__restrict__ Zimg)
{
    extern __shared__ float smz[];
    float *sG = smz;                        // sG[e * 129 + l] = (V^T V)(l, e)
    float *sY = sG + 128 * 129;             // sY[l * 65 + c]: Y, then Z
    float *sW = sY + 128 * 65;              // sW[l * 65 + c]
    float *sT = sW + 128 * 65;              // T_q(a, b) at q NB NB + a + b NB
    const int tid = threadIdx.x;
    const int64_t n_tr = n_ext - nbk;
    const int64_t cbase = (int64_t)blockIdx.x * BU_N;
    const int nq = (nbk + NB - 1) / NB;
    // G and Y as 16-byte vectors of Ysum (row e of the Gram matrix and column cg of Y are
    // 128 consecutive floats), each thread's loads all issued before its stores (a loop of
    // dependent load-store pairs left one L2 round trip per iteration exposed)
    {
        constexpr int GIT = 128 * 32 / 256;              // float4 of G per thread
        float4 gv[GIT];
#pragma unroll
        for (int it = 0; it < GIT; ++it) {
            const int idx = tid + it * 256, e = idx >> 5, l4 = (idx & 31) * 4;
            gv[it] = (e < nbk) ? __ldcg(reinterpret_cast<const float4 *>(Ysum + (int64_t)e * BK + l4))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        constexpr int YIT = BU_N * 32 / 256;             // float4 of Y per thread
        float4 yv[YIT];
#pragma unroll
        for (int it = 0; it < YIT; ++it) {
            const int idx = tid + it * 256, c = idx >> 5, l4 = (idx & 31) * 4;
            const int64_t cg = cbase + c;
            yv[it] = (cg < n_tr) ? __ldcg(reinterpret_cast<const float4 *>(Ysum + (nbk + cg) * BK + l4))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        asm volatile("" ::: "memory");                   // the loads above stay ahead of the stores
#pragma unroll
        for (int it = 0; it < GIT; ++it) {
            const int idx = tid + it * 256, e = idx >> 5, l4 = (idx & 31) * 4;
            float *d = sG + e * 129 + l4;
            d[0] = (l4 + 0 < e) ? gv[it].x : 0.f;
            d[1] = (l4 + 1 < e) ? gv[it].y : 0.f;
            d[2] = (l4 + 2 < e) ? gv[it].z : 0.f;
            d[3] = (l4 + 3 < e) ? gv[it].w : 0.f;
        }
#pragma unroll
        for (int it = 0; it < YIT; ++it) {
            const int idx = tid + it * 256, c = idx >> 5, l4 = (idx & 31) * 4;
            sY[(l4 + 0) * 65 + c] = (l4 + 0 < nbk) ? yv[it].x : 0.f;
            sY[(l4 + 1) * 65 + c] = (l4 + 1 < nbk) ? yv[it].y : 0.f;
            sY[(l4 + 2) * 65 + c] = (l4 + 2 < nbk) ? yv[it].z : 0.f;
            sY[(l4 + 3) * 65 + c] = (l4 + 3 < nbk) ? yv[it].w : 0.f;
        }
        const int nt4 = nq * NB * NB / 4;                // T blocks, a multiple of 4 floats
#pragma unroll 4
        for (int idx = tid; idx < nt4; idx += 256)
            reinterpret_cast<float4 *>(sT)[idx] = __ldg(reinterpret_cast<const float4 *>(Tb) + idx);
    }
    __syncthreads();
    // a thread's NB / 4 rows (l = q0 + g + 4 u) advance together, so that each step of
    // the sums reads Y (or W) once for all of them and the chains hide one another's
    // shared-memory latency (one chain at a time left about 30 us of exposed latency)
    const int c = tid & 63, g = tid >> 6;
    constexpr int NU = NB / 4;
    for (int q = 0; q < nq; ++q) {
        const int q0 = q * NB;
        float w[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) w[u] = sY[(q0 + g + 4 * u) * 65 + c];
#pragma unroll 4
        for (int l2 = 0; l2 < q0; ++l2) {
            const float y = sY[l2 * 65 + c];
#pragma unroll
            for (int u = 0; u < NU; ++u) w[u] -= sG[(q0 + g + 4 * u) * 129 + l2] * y;
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) sW[(q0 + g + 4 * u) * 65 + c] = w[u];
        __syncthreads();
        float z[NU];
#pragma unroll
        for (int u = 0; u < NU; ++u) z[u] = 0.f;
#pragma unroll
        for (int a = 0; a < NB; ++a) {
            const float wa = sW[(q0 + a) * 65 + c];
#pragma unroll
            for (int u = 0; u < NU; ++u) {
                const int b = g + 4 * u;
                if (a <= b) z[u] += sT[q * NB * NB + a + b * NB] * wa;
            }
        }
#pragma unroll
        for (int u = 0; u < NU; ++u) sY[(q0 + g + 4 * u) * 65 + c] = z[u];
        __syncthreads();
    }
    unsigned char *zi = Zimg + (int64_t)blockIdx.x * Z_TILE;
    for (int idx = tid; idx < BU_N * 16; idx += 256) {
        const int cc = idx >> 4, c16 = idx & 15, h = c16 >> 3, ch = c16 & 7;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int l = 8 * c16 + e;
            v[e] = (l < nq * NB) ? sY[l * 65 + cc] : 0.f;
        }
        uint4 p[3];
        split8(v, p);
        const uint32_t off = (uint32_t)cc * 128u + (((uint32_t)ch ^ ((uint32_t)cc & 7u)) << 4);
#pragma unroll
        for (int pp = 0; pp < 3; ++pp) *reinterpret_cast<uint4 *>(zi + (uint32_t)(h * 3 + pp) * ZPART + off) = p[pp];
    }
}

// ---------------------------------------------------------------------------
// k_bu: C(i, c) -= sum_l V(i, l) Z(l, c) for the trailing columns, rows k.. of F.
// Units (row tile r, column tile j) in row-tile-major order; CTA b takes a contiguous
// range.  Warp 0 loads the VU tile (when r changes) and the Z tiles (ring of two)
// (lane 0), and the unit's tile of C by TMA into one C buffer as soon as the epilogue
// has read the previous tile (lane 1); warp 1 issues the 48 MMAs of a unit into one of
// two TMEM buffers (the two K halves and the leading and small products in four
// accumulators, summed in the epilogue); warps 2..9 (two per lane quarter, 32 columns
// each) read their 32 elements of C from the C buffer and free it, read D, free the
// TMEM buffer, then store C - D.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BU_THREADS, 1)
k_bu(const __grid_constant__ CUtensorMap mC, float *__restrict__ F, int64_t ld, int64_t k, int nbk, int64_t mp,
     int64_t n_ext, const unsigned char *__restrict__ VU, const unsigned char *__restrict__ Zimg, int64_t j0,
     int64_t nj, int64_t n_units, int *flag)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = bt_align1024(smem_raw);
    unsigned char *VUs = base;
    const float *Cs = reinterpret_cast<const float *>(base + VU_TILE + 2 * Z_TILE);   // [64 columns][128 rows]
    __shared__ uint64_t vu_full, vu_empty, z_full[2], z_empty[2], acc_full[2], acc_empty[2], c_full, c_empty;
    __shared__ int s_vu_loads, s_last_z[2], s_last_commit, s_last_c;
    __shared__ volatile int s_fail;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u0 = (int64_t)blockIdx.x * n_units / gridDim.x;
    const int64_t u1 = ((int64_t)blockIdx.x + 1) * n_units / gridDim.x;
    const int nloc = (int)(u1 - u0);
    const int64_t n_tr = n_ext - nbk;

    if (warp == 0) tc::tmem_alloc(&tmem_slot, 512);
    if (threadIdx.x == 0) {
        tc::mbar_init(&vu_full, 1);
        tc::mbar_init(&vu_empty, 1);
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&z_full[s], 1);
            tc::mbar_init(&z_empty[s], 1);
            tc::mbar_init(&acc_full[s], 1);
            tc::mbar_init(&acc_empty[s], BU_EPI);
            s_last_z[s] = -1;
        }
        tc::mbar_init(&c_full, 1);
        tc::mbar_init(&c_empty, BU_EPI);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_vu_loads = 0;
        s_last_commit = -1;
        s_last_c = -1;
        s_fail = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int64_t prev_r = -1;
            int loads = 0;
            for (int lu = 0; lu < nloc; ++lu) {
                const int64_t u = u0 + lu, r = u / nj, j = j0 + u % nj;
                if (r != prev_r) {
                    if (loads > 0 && !tc::mbar_wait(&vu_empty, (uint32_t)(loads - 1) & 1u, BT_SPIN)) {
                        s_fail = 1;
                        break;
                    }
                    if (s_fail) break;
                    bt_expect_tx(&vu_full, VU_TILE);
                    bt_bulk_load(VUs, VU + r * VU_TILE, VU_TILE, &vu_full);
                    s_vu_loads = ++loads;
                    prev_r = r;
                }
                const int s = lu & 1;
                if (lu >= 2 && !tc::mbar_wait(&z_empty[s], (uint32_t)((lu - 2) >> 1) & 1u, BT_SPIN)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                bt_expect_tx(&z_full[s], Z_TILE);
                bt_bulk_load(base + VU_TILE + s * Z_TILE, Zimg + j * Z_TILE, Z_TILE, &z_full[s]);
                s_last_z[s] = lu;
            }
        } else if (lane == 1) {
            // the units' tiles of C by TMA into the one C buffer, once the epilogue has read
            // the previous tile out of it
            for (int lu = 0; lu < nloc; ++lu) {
                const int64_t u = u0 + lu, r = u / nj, j = j0 + u % nj;
                if (lu >= 1 && !tc::mbar_wait(&c_empty, (uint32_t)(lu - 1) & 1u, BT_SPIN)) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                bt_expect_tx(&c_full, BU_CT);
                bt_tma_2d(base + VU_TILE + 2 * Z_TILE, &mC, (int)(k + r * BU_R), (int)(k + nbk + j * BU_N), &c_full);
                s_last_c = lu;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16(BU_R, BU_N);
            int64_t prev_r = -1;
            int vu_idx = 0;
            uint64_t dA[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 0; p < 3; ++p) dA[h][p] = tc::smem_desc_sw128(VUs + (h * 3 + p) * PART128);
            for (int lu = 0; lu < nloc; ++lu) {
                const int64_t u = u0 + lu, r = u / nj;
                if (r != prev_r) {
                    if (!tc::mbar_wait(&vu_full, (uint32_t)vu_idx & 1u, BT_SPIN)) {
                        s_fail = 1;
                        break;
                    }
                    ++vu_idx;
                    prev_r = r;
                }
                const int s = lu & 1, b = lu & 1;
                if (!tc::mbar_wait(&z_full[s], (uint32_t)(lu >> 1) & 1u, BT_SPIN) ||
                    (lu >= 2 && !tc::mbar_wait(&acc_empty[b], (uint32_t)((lu - 2) >> 1) & 1u, BT_SPIN))) {
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                tc::fence_after_sync();
                const unsigned char *Zs = base + VU_TILE + s * Z_TILE;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // buffer b: [big h0 | big h1 | small h0 | small h1], BU_N columns each
                    const uint32_t dbig = tmem + (uint32_t)(256 * b + BU_N * h), dsmall = dbig + 2 * BU_N;
                    uint64_t dB[3];
#pragma unroll
                    for (int p = 0; p < 3; ++p) dB[p] = tc::smem_desc_sw128(Zs + (h * 3 + p) * ZPART);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t o = (uint64_t)(ks * 32) >> 4;
                        const uint32_t acc = ks > 0 ? 1u : 0u;
                        tc::mma_bf16(dbig, dA[h][0] + o, dB[0] + o, idesc, acc);
                        tc::mma_bf16(dsmall, dA[h][0] + o, dB[1] + o, idesc, acc);
                        tc::mma_bf16(dsmall, dA[h][1] + o, dB[0] + o, idesc, 1u);
                        tc::mma_bf16(dsmall, dA[h][0] + o, dB[2] + o, idesc, 1u);
                        tc::mma_bf16(dsmall, dA[h][2] + o, dB[0] + o, idesc, 1u);
                        tc::mma_bf16(dsmall, dA[h][1] + o, dB[1] + o, idesc, 1u);
                    }
                }
                tc::mma_commit(&z_empty[s]);
                tc::mma_commit(&acc_full[b]);
                const int64_t rn = (lu + 1 < nloc) ? (u + 1) / nj : -1;
                if (rn != r) tc::mma_commit(&vu_empty);
                s_last_commit = lu;
            }
        }
    } else {
        const int qd = warp & 3, hf = (warp - 2) >> 2;    // lane quarter, 32-column half
        for (int lu = 0; lu < nloc; ++lu) {
            const int64_t u = u0 + lu, r = u / nj, j = j0 + u % nj;
            const int b = lu & 1;
            // the thread's 32 elements of C first, from the TMA-loaded tile (which then
            // goes back to the loader for the next unit): they overlap the MMAs
            const int64_t i = r * BU_R + 32 * qd + lane;          // panel-local row
            const int64_t c0 = j * BU_N + 32 * hf;
            float *col = F + (k + i) + (k + nbk + c0) * ld;
            const int64_t nvalid = (i < mp) ? n_tr - c0 : 0;
            if (!tc::mbar_wait(&c_full, (uint32_t)lu & 1u, BT_SPIN)) {
                s_fail = 1;
                break;
            }
            float cv[32];
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) cv[jj] = Cs[(32 * hf + jj) * BU_R + 32 * qd + lane];
            __syncwarp();
            if (lane == 0) bt_arrive(&c_empty);
            if (!tc::mbar_wait(&acc_full[b], (uint32_t)(lu >> 1) & 1u, BT_SPIN)) {
                s_fail = 1;
                break;
            }
            if (s_fail) break;
            tc::fence_after_sync();
            float d[32];
#pragma unroll
            for (int cg = 0; cg < 2; ++cg) {
                float v0[16], v1[16], w0[16], w1[16];
                const uint32_t ta = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(256 * b + 32 * hf + 16 * cg);
                tc::tmem_ld16(ta, v0);
                tc::tmem_ld16(ta + BU_N, v1);
                tc::tmem_ld16(ta + 2 * BU_N, w0);
                tc::tmem_ld16(ta + 3 * BU_N, w1);
#pragma unroll
                for (int jj = 0; jj < 16; ++jj) d[16 * cg + jj] = (v0[jj] + v1[jj]) + (w0[jj] + w1[jj]);
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) bt_arrive(&acc_empty[b]);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
                if (jj < nvalid) col[(int64_t)jj * ld] = cv[jj] - d[jj];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (s_fail) {
        if (threadIdx.x == 0) {
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
            if (s_vu_loads > 0) tc::mbar_wait(&vu_full, (uint32_t)(s_vu_loads - 1) & 1u, BT_SPIN);
            for (int s = 0; s < 2; ++s)
                if (s_last_z[s] >= 0) tc::mbar_wait(&z_full[s], (uint32_t)(s_last_z[s] >> 1) & 1u, BT_SPIN);
            const int lc = s_last_commit;
            if (lc >= 0) tc::mbar_wait(&acc_full[lc & 1], (uint32_t)(lc >> 1) & 1u, BT_SPIN);
            if (s_last_c >= 0) tc::mbar_wait(&c_full, (uint32_t)s_last_c & 1u, BT_SPIN);
        }
        __syncthreads();
    }
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

template <typename K>
cudaError_t bt_smem_attr(K kernel, size_t bytes)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

constexpr size_t bz_smem(int nb) { return sizeof(float) * (128 * 129 + 2 * 128 * 65 + (size_t)128 * nb); }

}  // namespace

// C <- H^T C for the outer block of nbk <= 128 columns at column k (inner panels of
// width nb in {16, 32}, their T factors from Tb on), C = F's columns k + nbk .. ntot.
// Returns 1 when the shape is not taken (alignment), the caller then updates panel by
// panel.
int fl_block_update_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int nbk,
                        int64_t ntot, int nb, const float *Tb, float *Gout, int split_next)
{
    FL_TRY(fl_block_join(ctx));           // the previous block's split update pass
    const int64_t mp = m_aug - k, n_ext = ntot - k, n_tr = n_ext - nbk;
    if (n_tr <= 0 || mp <= 0) return 0;
    if (nbk < 1 || nbk > BK || (nb != 16 && nb != 32) || ld % 4 != 0 || k % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(F) & 15u) != 0)
        return 1;
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = bt_smem_attr(k_bimg, BI_SMEM);
        if (e == cudaSuccess) e = bt_smem_attr(k_by, BY_SMEM);
        if (e == cudaSuccess) e = bt_smem_attr(k_bz<16>, bz_smem(16));
        if (e == cudaSuccess) e = bt_smem_attr(k_bz<32>, bz_smem(32));
        if (e == cudaSuccess) e = bt_smem_attr(k_bu, BU_SMEM);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "block-update attributes");
        attr_once.done(ctx->device);
    }
    const int64_t nch = fl_cdiv(mp, BY_KC), n_rt = fl_cdiv(mp, BU_R), n_ct = fl_cdiv(n_tr, BU_N);
    const int64_t ytiles = fl_cdiv(n_ext, BY_N);
    // one wave of Y-pass CTAs (one per SM), each streaming at least 4 chunks of rows
    const int64_t S = std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms / ytiles, nch / 4));
    unsigned char *VY = (unsigned char *)fl_ws(ctx, FL_WS_BLK_VY, (size_t)nch * VY_CHUNK);
    unsigned char *VU = (unsigned char *)fl_ws(ctx, FL_WS_BLK_VU, (size_t)n_rt * VU_TILE);
    float *Ypart = (float *)fl_ws(ctx, FL_WS_BLK_Y, sizeof(float) * (size_t)(S + 1) * n_ext * BK);
    unsigned char *Zimg = (unsigned char *)fl_ws(ctx, FL_WS_BLK_Z, (size_t)n_ct * Z_TILE);
    if (!VY || !VU || !Ypart || !Zimg) return FASTLSQ_ERR_NOMEM;
    float *Ysum = Ypart + (size_t)S * n_ext * BK;
    CUtensorMap mF, mC;
    if (!fl_encode_f32_map(&mF, F, ld, ntot, BY_KC, BY_N, false) ||
        !fl_encode_f32_map(&mC, F, ld, ntot, BU_R, BU_N, false))
        return 1;
    {
        FL_PROF(ctx, FASTLSQ_K_BLOCK_PREP);
        k_bimg<<<(unsigned)n_rt, 256, BI_SMEM, ctx->stream>>>(F, ld, k, nbk, mp, nch, VY, VU);
        FL_CHECK_LAUNCH(ctx, "block image");
    }
    {
        FL_PROF(ctx, FASTLSQ_K_BLOCK_Y);
        k_by<<<dim3((unsigned)ytiles, (unsigned)S), BY_THREADS, BY_SMEM, ctx->stream>>>(
            mF, F, ld, k, nbk, mp, n_ext, VY, nch, Ypart, ctx->d_flag);
        FL_CHECK_LAUNCH(ctx, "block Y pass");
    }
    {
        FL_PROF_N(ctx, FASTLSQ_K_BLOCK_PREP, 2);
        k_bsum<<<(unsigned)fl_cdiv(n_ext, 8), 256, 0, ctx->stream>>>(Ypart, (int)S, n_ext, Ysum);
        FL_CHECK_LAUNCH(ctx, "block Y sum");
        if (Gout) {      // the block's own columns of Y: its Gram matrix
            const cudaError_t e = cudaMemcpyAsync(Gout, Ysum, sizeof(float) * (size_t)nbk * BK,
                                                  cudaMemcpyDeviceToDevice, ctx->stream);
            if (e != cudaSuccess) return fl_cuda(ctx, e, "block Gram copy");
        }
        if (nb == 32)
            k_bz<32><<<(unsigned)n_ct, 256, bz_smem(32), ctx->stream>>>(Ysum, n_ext, nbk, Tb, Zimg);
        else
            k_bz<16><<<(unsigned)n_ct, 256, bz_smem(16), ctx->stream>>>(Ysum, n_ext, nbk, Tb, Zimg);
        FL_CHECK_LAUNCH(ctx, "block Z");
    }
    // the update pass over column tiles [j0, j0 + nj)
    auto update = [&](int64_t j0, int64_t nj) -> int {
        const int64_t units = n_rt * nj;
        const unsigned G = (unsigned)std::min<int64_t>(ctx->num_sms, units);
        FL_PROF(ctx, FASTLSQ_K_BLOCK_U);
        k_bu<<<G, BU_THREADS, BU_SMEM, ctx->stream>>>(mC, F, ld, k, nbk, mp, n_ext, VU, Zimg, j0, nj, units,
                                                      ctx->d_flag);
        FL_CHECK_LAUNCH(ctx, "block update");
        return 0;
    };
    const int64_t nj_next = BK / BU_N;            // the next outer block's columns
    if (!split_next || n_ct <= nj_next) return update(0, n_ct);
    // the next block's columns first, on the caller's stream; the rest on the second
    // auxiliary stream, joined back before the next block's update (fl_block_join)
    FL_TRY(update(0, nj_next));
    cudaError_t e = cudaEventRecord(ctx->ev_fork2, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux2_stream, ctx->ev_fork2, 0);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "block update fork");
    cudaStream_t main_stream = ctx->stream;
    ctx->stream = ctx->aux2_stream;
    const int rc = update(nj_next, n_ct - nj_next);
    if (rc == 0) e = cudaEventRecord(ctx->ev_join2, ctx->aux2_stream);
    ctx->stream = main_stream;
    FL_TRY(rc);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "block update join");
    ctx->join2_pending = 1;
    return 0;
}

int fl_block_join(fastlsq_ctx *ctx)
{
    if (!ctx->join2_pending) return 0;
    ctx->join2_pending = 0;
    const cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join2, 0);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "block update join");
    return 0;
}

// Q^T y for the two-level FP32 factor (Sec. 2.3's QR applied to a right-hand side: the
// refinement's Q^T r and the re-solves of a kept factor, App. G.5), one cooperative
// launch with one grid barrier per outer block of 128 columns instead of one per inner
// panel.
//
// An outer block's reflectors act as one block reflector H_b = I - V_b T_b V_b^T, with
// T_b (128 x 128, upper triangular) formed once per factor by k_block_t from the
// block's Gram matrix V_b^T V_b (a by-product of the tensor-core Y pass) and the inner
// panels' T: appending panel q to the panels before it gives
//     T(0:c, c:c+nb) = -T(0:c, 0:c) (V_{0:c}^T V_q) T_q,   c = q nb.
// k_apply_qb then takes, per block in order:
//   s = V_b^T y   (each CTA over its rows, CTA partials in global memory, grid barrier),
//   w = T_b^T s,
//   y -= V_b w    (each CTA on its rows).
// Each CTA stages its rows of V_b (unit lower trapezoid applied) and T_b in shared
// memory with bulk copies, so V is read from memory once per application.  Waits are
// bounded: on timeout the device flag is raised and the CTA leaves.
#include <algorithm>

#include "common.cuh"
#include "gridsync.cuh"
#include "qr.cuh"
#include "tc_common.cuh"

namespace {

constexpr int QB_BK = 128;                     // outer block width
constexpr int QB_THREADS = 256;
constexpr int QB_MAX_ROWS = 296;               // rows per CTA (shared-memory capacity)
constexpr int QB_MAX_CTAS = 160;               // CTAs whose partials one thread adds (8 groups x 20)
constexpr long long QB_SPIN = 2000000000ll;    // SM cycles (about a second) before a wait gives up

__device__ __forceinline__ void qb_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                 :: "r"(tc::smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void qb_bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 :: "r"(tc::smem_addr(dst)), "l"(src), "r"(bytes), "r"(tc::smem_addr(bar)) : "memory");
}

// ---------------------------------------------------------------------------
// k_block_t: T_b of outer block blockIdx.x from its Gram matrix (Gall: per block
// G[e * 128 + l] = v_l^T v_e) and the inner panels' T (Tall: per panel, T(q, l) at
// q + NB l).  Output per block row-major: Tball[q * 128 + l] = T_b(q, l), zero outside
// the block's columns.
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(256)
k_block_t(const float *__restrict__ Gall, const float *__restrict__ Tall, int64_t n, float *__restrict__ Tball)
{
    extern __shared__ float smb[];
    float *Gs = smb;                        // [128][129]: Gs[l * 129 + e] = v_l^T v_e
    float *Ts = Gs + QB_BK * 129;           // [128][129]: Ts[q * 129 + l] = T_b(q, l)
    float *X = Ts + QB_BK * 129;            // [128][NB + 1]
    const int b = blockIdx.x;
    const int64_t kb = (int64_t)b * QB_BK;
    const int nbk = (int)fl_min64(QB_BK, n - kb);
    const int npan = (nbk + NB - 1) / NB;
    const float *G = Gall + (int64_t)b * QB_BK * QB_BK;
    for (int idx = threadIdx.x; idx < QB_BK * QB_BK; idx += blockDim.x) {
        const int e = idx / QB_BK, l = idx % QB_BK;
        Gs[l * 129 + e] = (l < nbk && e < nbk) ? G[idx] : 0.f;
        Ts[(idx / QB_BK) * 129 + idx % QB_BK] = 0.f;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < npan * NB * NB; idx += blockDim.x) {
        const int p = idx / (NB * NB), r = idx % (NB * NB), q = r % NB, l = r / NB;
        if (p * NB + q < nbk && p * NB + l < nbk)
            Ts[(p * NB + q) * 129 + p * NB + l] = Tall[(kb / NB + p) * NB * NB + q + NB * l];
    }
    __syncthreads();
    for (int q = 1; q < npan; ++q) {
        const int c0 = q * NB;
        // X = (V_{0:c0}^T V_q) T_q   (c0 x NB; T_q upper triangular)
        for (int idx = threadIdx.x; idx < c0 * NB; idx += blockDim.x) {
            const int i = idx / NB, j = idx % NB;
            float x = 0.f;
            for (int t = 0; t <= j; ++t) x = fmaf(Gs[i * 129 + c0 + t], Ts[(c0 + t) * 129 + c0 + j], x);
            X[i * (NB + 1) + j] = x;
        }
        __syncthreads();
        // T(0:c0, c0:c0+NB) = -T(0:c0, 0:c0) X   (T(0:c0, 0:c0) upper triangular)
        for (int idx = threadIdx.x; idx < c0 * NB; idx += blockDim.x) {
            const int i = idx / NB, j = idx % NB;
            float acc = 0.f;
            for (int i2 = i; i2 < c0; ++i2) acc = fmaf(Ts[i * 129 + i2], X[i2 * (NB + 1) + j], acc);
            Ts[i * 129 + c0 + j] = -acc;
        }
        __syncthreads();
    }
    float *out = Tball + (int64_t)b * QB_BK * QB_BK;
    for (int idx = threadIdx.x; idx < QB_BK * QB_BK; idx += blockDim.x)
        out[idx] = Ts[(idx / QB_BK) * 129 + idx % QB_BK];
}

// Shared memory of k_apply_qb (offsets in floats; every piece starts on 16 bytes)
struct QbLayout {
    int pr;                                   // column pitch of the staged rows, = 4 mod 8
    __host__ __device__ explicit QbLayout(int p) : pr(p) {}
    __host__ __device__ size_t Vs() const { return 0; }                        // [128][pr]
    __host__ __device__ size_t Ts() const { return (size_t)QB_BK * pr; }       // [128 * 128]
    __host__ __device__ size_t ys() const { return Ts() + QB_BK * QB_BK; }     // [pr]
    __host__ __device__ size_t sv() const { return ys() + pr; }                // [128]
    __host__ __device__ size_t wv() const { return sv() + QB_BK; }             // [128]
    __host__ __device__ size_t red() const { return wv() + QB_BK; }            // [8][128]
    __host__ __device__ size_t bytes() const { return sizeof(float) * (red() + 8 * QB_BK); }
};

__global__ void __launch_bounds__(QB_THREADS, 1)
k_apply_qb(const float *__restrict__ F, int64_t ld, int64_t m_aug, int64_t n, const float *__restrict__ Tball,
           float *__restrict__ y, int rpc, int pr, float *__restrict__ part, GridBar *bar, int *flag)
{
    extern __shared__ __align__(16) float sq[];
    __shared__ uint64_t lbar;
    __shared__ volatile int s_abort;
    const QbLayout L(pr);
    float *Vs = sq + L.Vs(), *Ts = sq + L.Ts(), *ys = sq + L.ys(), *sv = sq + L.sv(), *wv = sq + L.wv();
    float *red = sq + L.red();
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x;
    const int64_t r_lo = (int64_t)blockIdx.x * rpc;
    const int64_t r_hi = fl_min64(m_aug, r_lo + rpc);
    const int nrow = (int)fl_max64(0, r_hi - r_lo);
    if (tid == 0) {
        tc::mbar_init(&lbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
    }
    for (int j = tid; j < pr; j += QB_THREADS) ys[j] = (j < nrow) ? y[r_lo + j] : 0.f;
    __syncthreads();
    const int nblk = (int)((n + QB_BK - 1) / QB_BK);
    int waits = 0;                                     // completed phases of lbar
    for (int st = 0; st < nblk; ++st) {
        const int b = st;
        const int par = st & 1;
        const int64_t kb = (int64_t)b * QB_BK;
        const int nbk = (int)fl_min64(QB_BK, n - kb);
        const int64_t r0 = fl_max64(r_lo, kb);         // first row of V_b here (a multiple of 4)
        const int nv = (int)fl_max64(0, r_hi - r0);    // staged rows
        const int nv4 = (nv + 3) & ~3;                 // whole 16-byte granules (F's rows are padded)
        const int off = (int)(r0 - r_lo);              // the staged rows' offset in ys
        if (tid == 0) {
            qb_expect_tx(&lbar, (uint32_t)(nbk * nv4 * 4 + QB_BK * QB_BK * 4));
            if (nv4 > 0)
                for (int c = 0; c < nbk; ++c)
                    qb_bulk_load(Vs + (size_t)c * pr, F + r0 + (kb + c) * ld, (uint32_t)nv4 * 4u, &lbar);
            qb_bulk_load(Ts, Tball + (int64_t)b * QB_BK * QB_BK, QB_BK * QB_BK * 4u, &lbar);
        }
        if (!tc::mbar_wait(&lbar, (uint32_t)(waits & 1), QB_SPIN)) {
            s_abort = 1;
            atomicCAS(flag, 0, FL_DEVERR_TIMEOUT);
        }
        ++waits;
        // V_b's unit lower trapezoid on the rows kb .. kb + nbk - 1; the padding rows zero
        const int jt = (int)fl_max64(0, fl_min64(nv, kb + nbk - r0));
        for (int idx = tid; idx < nbk * jt; idx += QB_THREADS) {
            const int c = idx / jt, j = idx % jt;
            const int64_t d = r0 + j - kb;             // row within the block
            if (d <= c) Vs[(size_t)c * pr + j] = (d == c) ? 1.f : 0.f;
        }
        for (int idx = tid; idx < nbk * (nv4 - nv); idx += QB_THREADS)
            Vs[(size_t)(idx / (nv4 - nv)) * pr + nv + idx % (nv4 - nv)] = 0.f;
        __syncthreads();
        if (s_abort) break;                            // uniform after the barrier
        // s partials: thread (c, h) adds rows 4h.., in steps of 8 rows, of column c
        {
            const int c = tid & (QB_BK - 1), h = tid >> 7;
            float a0 = 0.f, a1 = 0.f;
            if (c < nbk)
                for (int j = 4 * h; j < nv4; j += 8) {
                    const float4 v = *reinterpret_cast<const float4 *>(Vs + (size_t)c * pr + j);
                    const float4 u = *reinterpret_cast<const float4 *>(ys + off + j);
                    a0 = fmaf(v.x, u.x, a0);
                    a1 = fmaf(v.y, u.y, a1);
                    a0 = fmaf(v.z, u.z, a0);
                    a1 = fmaf(v.w, u.w, a1);
                }
            red[h * QB_BK + c] = a0 + a1;
        }
        __syncthreads();
        if (tid < QB_BK) __stcg(part + ((int64_t)par * G + blockIdx.x) * QB_BK + tid, red[tid] + red[QB_BK + tid]);
        if (!grid_sync(bar, G, flag, &s_abort)) break;
        // s = the CTAs' partials added in a fixed order: thread (group g, column quad cq)
        // adds CTAs g, g + 8, ... (all loads in flight at once), then the 8 groups in order
        {
            const int cq = tid & 31, g = tid >> 5;
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 v[QB_MAX_CTAS / 8];
#pragma unroll
            for (int i = 0; i < QB_MAX_CTAS / 8; ++i) {
                const unsigned cta = (unsigned)(g + 8 * i);
                v[i] = (cta < G) ? __ldcg(reinterpret_cast<const float4 *>(part + ((int64_t)par * G + cta) * QB_BK) + cq)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < QB_MAX_CTAS / 8; ++i) {
                acc.x += v[i].x;
                acc.y += v[i].y;
                acc.z += v[i].z;
                acc.w += v[i].w;
            }
            *reinterpret_cast<float4 *>(red + g * QB_BK + 4 * cq) = acc;
        }
        __syncthreads();
        if (tid < QB_BK) {
            float s = 0.f;
#pragma unroll
            for (int g = 0; g < 8; ++g) s += red[g * QB_BK + tid];
            sv[tid] = (tid < nbk) ? s : 0.f;
        }
        __syncthreads();
        // w = T_b^T s; T_b(q, l) at Ts[q * 128 + l]
        if (tid < QB_BK) {
            float acc = 0.f;
            for (int q = 0; q <= tid; ++q) acc = fmaf(Ts[q * QB_BK + tid], sv[q], acc);
            wv[tid] = acc;
        }
        __syncthreads();
        // y -= V_b w on the staged rows
        for (int j = tid; j < nv; j += QB_THREADS) {
            float a0 = 0.f, a1 = 0.f;
            int c = 0;
            for (; c + 1 < nbk; c += 2) {
                a0 = fmaf(Vs[(size_t)c * pr + j], wv[c], a0);
                a1 = fmaf(Vs[(size_t)(c + 1) * pr + j], wv[c + 1], a1);
            }
            if (c < nbk) a0 = fmaf(Vs[(size_t)c * pr + j], wv[c], a0);
            ys[off + j] -= a0 + a1;
        }
        __syncthreads();
    }
    if (s_abort) {
        // a timed-out wait: let this CTA's own copies land before the CTA leaves
        if (tid == 0 && waits > 0) tc::mbar_wait(&lbar, (uint32_t)((waits - 1) & 1), QB_SPIN);
        __syncthreads();
        return;
    }
    for (int j = tid; j < nrow; j += QB_THREADS) y[r_lo + j] = ys[j];
}

// rows per CTA and the staged pitch for m_aug rows on G CTAs; false when too tall
bool qb_shape(int64_t m_aug, int G, int &rpc, int &pr)
{
    rpc = (int)fl_round_up(fl_cdiv(m_aug, G), 4);
    if (rpc > QB_MAX_ROWS) return false;
    pr = (rpc % 8 == 0) ? rpc + 4 : rpc;     // = 4 mod 8: conflict-free 16-byte column reads
    return true;
}

}  // namespace

int fl_block_t_f32(fastlsq_ctx *ctx, const float *Gall, const float *Tall, int64_t n, int nb, float *Tball)
{
    const size_t smem = sizeof(float) * ((size_t)2 * QB_BK * 129 + (size_t)QB_BK * (nb + 1));
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_block_t<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(float) * (2 * QB_BK * 129 + QB_BK * 33)));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_block_t<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(float) * (2 * QB_BK * 129 + QB_BK * 33)));
        if (e != cudaSuccess) return fl_cuda(ctx, e, "block T attributes");
        attr_once.done(ctx->device);
    }
    const unsigned nblk = (unsigned)fl_cdiv(n, QB_BK);
    FL_PROF(ctx, FASTLSQ_K_BLOCK_PREP);
    if (nb == 16) k_block_t<16><<<nblk, 256, smem, ctx->stream>>>(Gall, Tall, n, Tball);
    else if (nb == 32) k_block_t<32><<<nblk, 256, smem, ctx->stream>>>(Gall, Tall, n, Tball);
    else return fl_fail(ctx, FASTLSQ_ERR_INVALID, "panel width %d", nb);
    FL_CHECK_LAUNCH(ctx, "block T");
    return 0;
}

int fl_apply_qb_f32(fastlsq_ctx *ctx, const float *F, int64_t ld, int64_t m_aug, int64_t n, const float *Tball,
                    float *y, int transpose)
{
    if (!transpose || ld % 4 != 0 || (reinterpret_cast<uintptr_t>(F) & 15u) != 0) return 1;
    const int G = std::min(ctx->num_sms, QB_MAX_CTAS);
    int rpc, pr;
    if (!qb_shape(m_aug, G, rpc, pr)) return 1;
    const QbLayout L(pr);
    const size_t smem = L.bytes();
    const size_t cap = (size_t)ctx->max_smem_optin - 1024;
    if (smem > cap) return 1;
    static FlOncePerDevice attr_once;
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_apply_qb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "apply_qb attributes");
        attr_once.done(ctx->device);
    }
    float *part = (float *)fl_ws(ctx, FL_WS_APPLYQ, sizeof(float) * 2 * (size_t)G * QB_BK);
    if (!part) return FASTLSQ_ERR_NOMEM;
    GridBar *bar = (GridBar *)ctx->d_grid_bar;
    int *flag = ctx->d_flag;
    void *args[] = {(void *)&F, (void *)&ld, (void *)&m_aug, (void *)&n, (void *)&Tball, (void *)&y,
                    (void *)&rpc, (void *)&pr, (void *)&part, (void *)&bar, (void *)&flag};
    FL_PROF(ctx, FASTLSQ_K_APPLY_Q);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_apply_qb, dim3((unsigned)G), dim3(QB_THREADS),
                                                args, smem, ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "apply_qb launch");
    return 0;
}

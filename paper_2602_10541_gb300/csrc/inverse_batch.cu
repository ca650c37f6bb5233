// Batched inverse problem with pre-factored operators (Sec. 3.8 in steady form;
// Sec. 2.5: gradients through the pre-factored solve, two triangular solves per
// evaluation): many instances of uneven size, every gradient evaluation of the whole
// batch in ONE persistent launch.
//
// fastlsq_inverse_prepare factors each instance once (FP64 Householder QR of
// [A; sqrt(mu) I], kept: the checkpoint the evaluations reuse) and tabulates its
// sensor matrix H_s (n_sens x n_feat, FP64).  fastlsq_inverse_eval launches
// k_inv_eval: a grid of persistent CTAs that take instances from a device-side queue
// (one atomic counter, instances in decreasing order of m_aug n, so the longest start
// first); one CTA runs an instance's whole evaluation with its vectors in shared memory:
//   y   = [s(x_int; theta); 0 (u = 0 rows); 0 (sqrt(mu) rows)]
//   y  <- Q^T y                       (the factor's reflectors, panel by panel)
//   beta = R^{-1} y[0:n]              (blocked substitution)
//   u_s = H_s beta, L = mean (u_s - y_obs)^2, g = dL/du_s
//   w   = R^{-T} (H_s^T g)
//   z   = Q [w; 0]                    (= A (A^T A + mu I)^{-1} H_s^T g = dL/d rhs)
//   dL/dtheta = sum_{i < n_int} z_i ds(x_i; theta)/dtheta
// No CTA waits on another: the queue is the only shared state, so nothing needs a
// timeout.  The launch allocates nothing and synchronises nothing on the host, so a
// caller can capture it in a CUDA graph and replay it with new theta and y_obs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "qr.cuh"

namespace {

constexpr int IB_MAX_SRC = 8;
constexpr int IB_MAX_SENS = 256;
constexpr int IB_NB = 32;              // largest panel width of an FP64 factor

struct InvDesc {
    int64_t n_int, n_feat, n_sens, m_aug, ld;
    int nb;
    double scale;
    const double *x_int, *theta, *y_obs, *H;      // H: [n_sens][n_feat]
    const double *F, *T;                          // factor (V below, R above), T blocks
    double *beta, *loss, *dtheta;
};

// sensor matrix H[s][j] = scale sin(W_j . x_s + b_j) (the features at the sensors), FP64
__global__ void k_sensor_matrix(const double *__restrict__ xs, int64_t ns, const double *__restrict__ W,
                                const double *__restrict__ b, int64_t n, double scale, double *__restrict__ H)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = blockIdx.y;
    if (j >= n) return;
    const double z = W[2 * j] * xs[2 * s] + W[2 * j + 1] * xs[2 * s + 1] + b[j];
    H[s * n + j] = scale * sin(z);
}

// lane l returns the warp's sum of vals[l]
__device__ __forceinline__ double ib_reduce_scatter(double (&vals)[IB_NB], int lane)
{
#pragma unroll
    for (int s = IB_NB / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int q = 0; q < s; ++q) {
            const double send = up ? vals[q] : vals[q + s];
            const double keep = up ? vals[q + s] : vals[q];
            vals[q] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return vals[0];
}

// y <- Q^T y (transpose) or Q y on the CTA's shared vector y[0, m_aug), FP64.  Per
// panel: s = V^T y (each thread its rows, warp reduce-scatter, warps summed in order),
// w = T^T s or T s, y -= V w.
template <int THREADS>
__device__ void ib_apply_q(const InvDesc &D, double *y, double *red, double *wv, bool transpose)
{
    constexpr int NW = THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = D.n_feat, m_aug = D.m_aug, ld = D.ld;
    const int nb = D.nb;
    const int P = (int)((n + nb - 1) / nb);
    for (int step = 0; step < P; ++step) {
        const int p = transpose ? step : P - 1 - step;
        const int64_t k = (int64_t)p * nb;
        const int nc = (int)fl_min64(nb, n - k);
        double acc[IB_NB];
#pragma unroll
        for (int l = 0; l < IB_NB; ++l) acc[l] = 0.0;
        for (int64_t i = k + tid; i < m_aug; i += THREADS) {
            const double yi = y[i];
            const int64_t li = i - k;
            const double *row = D.F + i + k * ld;
            if (li >= IB_NB) {
#pragma unroll
                for (int l = 0; l < IB_NB; ++l)
                    if (l < nc) acc[l] = fma(row[(int64_t)l * ld], yi, acc[l]);
            } else {
#pragma unroll
                for (int l = 0; l < IB_NB; ++l) {
                    const double v = (l >= nc || li < l) ? 0.0 : (li == l ? 1.0 : row[(int64_t)l * ld]);
                    acc[l] = fma(v, yi, acc[l]);
                }
            }
        }
        const double part = ib_reduce_scatter(acc, lane);
        red[warp * IB_NB + lane] = part;
        __syncthreads();
        if (warp == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) s += red[w * IB_NB + lane];
            const double *T = D.T + (int64_t)p * nb * nb;      // T(q, l) at q + l nb
            double wl = 0.0;
            for (int q = 0; q < nc; ++q) {
                const double sq = __shfl_sync(0xffffffffu, s, q);
                if (lane < nc) {
                    if (transpose) { if (q <= lane) wl = fma(T[q + (int64_t)lane * nb], sq, wl); }
                    else { if (q >= lane) wl = fma(T[lane + (int64_t)q * nb], sq, wl); }
                }
            }
            wv[lane] = (lane < nc) ? wl : 0.0;
        }
        __syncthreads();
        for (int64_t i = k + tid; i < m_aug; i += THREADS) {
            const int64_t li = i - k;
            const double *row = D.F + i + k * ld;
            double s = 0.0;
            if (li >= IB_NB) {
#pragma unroll
                for (int l = 0; l < IB_NB; ++l)
                    if (l < nc) s = fma(row[(int64_t)l * ld], wv[l], s);
            } else {
#pragma unroll
                for (int l = 0; l < IB_NB; ++l) {
                    const double v = (l >= nc || li < l) ? 0.0 : (li == l ? 1.0 : row[(int64_t)l * ld]);
                    s = fma(v, wv[l], s);
                }
            }
            y[i] -= s;
        }
        __syncthreads();
    }
}

// x <- R^{-1} x (transpose = false) or R^{-T} x on the CTA's shared vector x[0, n),
// R the upper triangle of the factor; blocks of 32 columns: warp 0 solves the
// diagonal block from registers (shuffles), then every thread updates the rest.
template <int THREADS>
__device__ void ib_trsv(const InvDesc &D, double *x, bool transpose)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = D.n_feat, ld = D.ld;
    const double *F = D.F;
    const int nblk = (int)((n + 31) / 32);
    for (int st = 0; st < nblk; ++st) {
        const int jb = transpose ? st : nblk - 1 - st;
        const int64_t c0 = (int64_t)jb * 32, c1 = fl_min64(n, c0 + 32);
        const int bw = (int)(c1 - c0);
        if (warp == 0) {
            // lane t holds x[c0 + t] and, for the solve, a row (no transpose: R(c0 + t, c0 + i))
            // or a column (transpose: R(c0 + i, c0 + t)) of the diagonal block
            double rr[32];
            double xv = (lane < bw) ? x[c0 + lane] : 0.0;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                rr[i] = 0.0;
                if (lane < bw && i < bw)
                    rr[i] = transpose ? F[(c0 + i) + (c0 + lane) * ld] : F[(c0 + lane) + (c0 + i) * ld];
            }
            if (!transpose) {
#pragma unroll
                for (int c = 31; c >= 0; --c) {
                    if (c >= bw) continue;
                    double xc = 0.0;
                    if (lane == c) xc = xv / rr[c];
                    xc = __shfl_sync(0xffffffffu, xc, c);
                    if (lane == c) xv = xc;
                    if (lane < c) xv = fma(-rr[c], xc, xv);
                }
            } else {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    if (r >= bw) continue;
                    double xr = 0.0;
                    if (lane == r) xr = xv / rr[r];
                    xr = __shfl_sync(0xffffffffu, xr, r);
                    if (lane == r) xv = xr;
                    if (lane > r) xv = fma(-rr[r], xr, xv);
                }
            }
            if (lane < bw) x[c0 + lane] = xv;
        }
        __syncthreads();
        if (!transpose) {
            for (int64_t r = tid; r < c0; r += THREADS) {       // rows above the block
                double s = 0.0;
                for (int i = 0; i < bw; ++i) s = fma(F[r + (c0 + i) * ld], x[c0 + i], s);
                x[r] -= s;
            }
        } else {
            for (int64_t c = c1 + tid; c < n; c += THREADS) {   // columns right of the block
                const double *col = F + c * ld;
                double s = 0.0;
                for (int i = 0; i < bw; ++i) s = fma(col[c0 + i], x[c0 + i], s);
                x[c] -= s;
            }
        }
        __syncthreads();
    }
}

// sum over the CTA of v (fixed order: warps in order), returned to every thread
template <int THREADS>
__device__ double ib_block_sum(double v, double *red)
{
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += red[w];
    return s;
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
k_inv_eval(const InvDesc *__restrict__ descs, const int *__restrict__ order, int n_inst,
           int *__restrict__ queue, int n_src, int64_t m_aug_max, int64_t n_max)
{
    constexpr int NW = THREADS / 32;
    extern __shared__ double ib_sm[];
    double *y = ib_sm;                          // [m_aug_max]
    double *xv = y + m_aug_max;                 // [n_max]
    double *red = xv + n_max;                   // [NW][32]
    double *wv = red + NW * IB_NB;              // [32]
    double *gs = wv + IB_NB;                    // [IB_MAX_SENS]
    double *th = gs + IB_MAX_SENS;              // [4 IB_MAX_SRC]
    __shared__ int s_q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) s_q = atomicAdd(queue, 1);
        __syncthreads();
        const int q = s_q;
        if (q >= n_inst) break;
        const InvDesc D = descs[order[q]];
        const int64_t n = D.n_feat;
        for (int t = tid; t < 4 * n_src; t += THREADS) th[t] = D.theta[t];
        __syncthreads();
        // source at the interior rows, zero elsewhere
        for (int64_t i = tid; i < D.m_aug; i += THREADS) {
            double v = 0.0;
            if (i < D.n_int) {
                const double px = D.x_int[2 * i], py = D.x_int[2 * i + 1];
                for (int s = 0; s < n_src; ++s) {
                    const double dx = px - th[4 * s], dy = py - th[4 * s + 1], w = th[4 * s + 2];
                    v += th[4 * s + 3] * exp(-(dx * dx + dy * dy) / (2.0 * w * w));
                }
            }
            y[i] = v;
        }
        __syncthreads();
        ib_apply_q<THREADS>(D, y, red, wv, true);
        for (int64_t j = tid; j < n; j += THREADS) xv[j] = y[j];
        __syncthreads();
        ib_trsv<THREADS>(D, xv, false);                          // beta
        for (int64_t j = tid; j < n; j += THREADS) D.beta[j] = xv[j];
        // sensors: warp per sensor, lanes over features
        for (int64_t s = warp; s < D.n_sens; s += NW) {
            const double *h = D.H + s * n;
            double u = 0.0;
            for (int64_t j = lane; j < n; j += 32) u = fma(h[j], xv[j], u);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
            if (lane == 0) gs[s] = u - D.y_obs[s];
        }
        __syncthreads();
        double l2 = 0.0;
        for (int64_t s = tid; s < D.n_sens; s += THREADS) l2 += gs[s] * gs[s];
        l2 = ib_block_sum<THREADS>(l2, red);
        if (tid == 0) *D.loss = l2 / (double)D.n_sens;
        for (int64_t s = tid; s < D.n_sens; s += THREADS) gs[s] *= 2.0 / (double)D.n_sens;
        __syncthreads();
        // grad_beta = H_s^T g, then w = R^{-T} grad_beta
        for (int64_t j = tid; j < n; j += THREADS) {
            double a = 0.0;
            for (int64_t s = 0; s < D.n_sens; ++s) a = fma(D.H[s * n + j], gs[s], a);
            xv[j] = a;
        }
        __syncthreads();
        ib_trsv<THREADS>(D, xv, true);
        // z = Q [w; 0]
        for (int64_t i = tid; i < D.m_aug; i += THREADS) y[i] = (i < n) ? xv[i] : 0.0;
        __syncthreads();
        ib_apply_q<THREADS>(D, y, red, wv, false);
        // dL/dtheta = sum over the interior rows of z_i ds(x_i)/dtheta
        double acc[4 * IB_MAX_SRC];
#pragma unroll
        for (int t = 0; t < 4 * IB_MAX_SRC; ++t) acc[t] = 0.0;
        for (int64_t i = tid; i < D.n_int; i += THREADS) {
            const double px = D.x_int[2 * i], py = D.x_int[2 * i + 1], zi = y[i];
#pragma unroll
            for (int s = 0; s < IB_MAX_SRC; ++s) {
                if (s >= n_src) break;
                const double *t = th + 4 * s;
                const double dx = px - t[0], dy = py - t[1];
                const double r2 = dx * dx + dy * dy, w2 = t[2] * t[2];
                const double e = exp(-r2 / (2.0 * w2));
                acc[4 * s + 0] = fma(zi * t[3] * e, dx / w2, acc[4 * s + 0]);
                acc[4 * s + 1] = fma(zi * t[3] * e, dy / w2, acc[4 * s + 1]);
                acc[4 * s + 2] = fma(zi * t[3] * e, r2 / (w2 * t[2]), acc[4 * s + 2]);
                acc[4 * s + 3] = fma(zi, e, acc[4 * s + 3]);
            }
        }
#pragma unroll
        for (int t = 0; t < 4 * IB_MAX_SRC; ++t) {
            if (t >= 4 * n_src) break;                   // uniform over the CTA
            const double v = ib_block_sum<THREADS>(acc[t], red);
            if (tid == 0) D.dtheta[t] = v;
        }
        __syncthreads();
    }
}

size_t ib_smem(int threads, int64_t m_aug_max, int64_t n_max)
{
    return sizeof(double) * ((size_t)m_aug_max + (size_t)n_max + (size_t)(threads / 32) * IB_NB + IB_NB +
                             IB_MAX_SENS + 4 * IB_MAX_SRC);
}

}  // namespace

struct fastlsq_inverse_plan {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_inst = 0, n_src = 0;
    int64_t m_aug_max = 0, n_max = 0;
    std::vector<fastlsq_factor *> factors;
    double *H = nullptr;          // sensor matrices, all instances
    InvDesc *d_desc = nullptr;
    int *d_order = nullptr;
    int *d_queue = nullptr;
    std::vector<InvDesc> h_desc;
    std::vector<int> h_order;
};

namespace {

template <int THREADS>
cudaError_t ib_launch(const fastlsq_inverse_plan *P, cudaStream_t st, int grid, size_t smem)
{
    static FlOncePerDevice once;
    if (once.pending(P->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_inv_eval<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        // a later plan may need more: set the largest the device allows
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
        e = cudaFuncSetAttribute(k_inv_eval<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 1024);
        if (e != cudaSuccess) return e;
        once.done(P->device);
    }
    k_inv_eval<THREADS><<<grid, THREADS, smem, st>>>(P->d_desc, P->d_order, P->n_inst, P->d_queue, P->n_src,
                                                     P->m_aug_max, P->n_max);
    return cudaGetLastError();
}

void plan_free(fastlsq_inverse_plan *P)
{
    if (!P) return;
    for (fastlsq_factor *f : P->factors) fastlsq_factor_destroy(f);
    if (P->H) cudaFreeAsync(P->H, P->stream);
    if (P->d_desc) cudaFreeAsync(P->d_desc, P->stream);
    if (P->d_order) cudaFreeAsync(P->d_order, P->stream);
    if (P->d_queue) cudaFreeAsync(P->d_queue, P->stream);
    delete P;
}

}  // namespace

extern "C" int fastlsq_inverse_prepare(fastlsq_ctx *ctx, const fastlsq_inverse_instance *inst, int32_t n_inst,
                                       const fastlsq_op *op, int32_t n_src, const fastlsq_inverse_opts *o,
                                       fastlsq_inverse_plan **out)
{
    if (!ctx || !out) return FASTLSQ_ERR_INVALID;
    *out = nullptr;
    if (!inst || !op || !o || n_inst < 1) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_prepare: bad arguments");
    if (n_src < 1 || n_src > IB_MAX_SRC)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_prepare: n_src 1..%d", IB_MAX_SRC);
    if (!(o->mu > 0) || !std::isfinite(o->mu))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_prepare: mu must be positive");
    fl_op_params opL;
    FL_TRY(fl_pack_op(ctx, op, &opL));
    if (opL.d != 2 || opL.n_pp != 0)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_prepare: 2-D operator without per-point terms");
    fl_op_params opI;
    memset(&opI, 0, sizeof(opI));
    opI.d = 2;
    opI.n_terms = 1;
    opI.coef[0] = 1.0;
    int64_t m_max = 0, n_max = 0, maug_max = 0;
    for (int q = 0; q < n_inst; ++q) {
        const fastlsq_inverse_instance &I = inst[q];
        if (I.n_int < 1 || I.n_bc < 0 || I.n_feat < 1 || I.n_feat > FL_MAX_FEAT || I.n_sens < 1 ||
            I.n_sens > IB_MAX_SENS || !I.x_int || (I.n_bc && !I.x_bc) || !I.W || !I.b || !I.sensors || !I.y_obs ||
            !I.theta || !I.beta || !I.loss || !I.dtheta)
            return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_prepare: bad instance %d", q);
        m_max = std::max<int64_t>(m_max, fl_round_up(I.n_int + I.n_bc, 4));
        n_max = std::max<int64_t>(n_max, I.n_feat);
        maug_max = std::max<int64_t>(maug_max, I.n_int + I.n_bc + I.n_feat);
    }
    // the evaluation keeps y [m_aug] and one n-vector per CTA in shared memory
    if (ib_smem(512, maug_max, n_max) > (size_t)ctx->max_smem_optin - 1024)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID,
                       "inverse_prepare: %lld rows + features exceed the evaluation's shared memory",
                       (long long)maug_max);
    fastlsq_inverse_plan *P = new (std::nothrow) fastlsq_inverse_plan();
    if (!P) return FASTLSQ_ERR_NOMEM;
    P->device = ctx->device;
    P->stream = ctx->stream;
    P->n_inst = n_inst;
    P->n_src = n_src;
    P->m_aug_max = maug_max;
    P->n_max = n_max;
    P->factors.assign(n_inst, nullptr);
    P->h_desc.resize(n_inst);
    size_t h_total = 0;
    for (int q = 0; q < n_inst; ++q) h_total += (size_t)inst[q].n_sens * inst[q].n_feat;
    double *A64 = nullptr, *pref = nullptr;
    cudaError_t e = cudaMallocAsync(&A64, sizeof(double) * m_max * n_max, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&pref, sizeof(double) * (2 + FL_MAX_PP) * n_max, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P->H, sizeof(double) * h_total, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P->d_desc, sizeof(InvDesc) * n_inst, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P->d_order, sizeof(int) * n_inst, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P->d_queue, sizeof(int), ctx->stream);
    int rc = (e == cudaSuccess) ? 0 : fl_cuda(ctx, e, "inverse_prepare buffers");
    size_t h_off = 0;
    for (int q = 0; q < n_inst && rc >= 0; ++q) {
        const fastlsq_inverse_instance &I = inst[q];
        const int64_t n = I.n_feat, m = I.n_int + I.n_bc, ld = fl_round_up(m, 4);
        const double scale = 1.0 / sqrt((double)n);
        do {
            if ((rc = fl_prefactors(ctx, opL, I.W, n, scale, 1.0, pref)) < 0) break;
            if ((rc = fl_launch_assemble_f64(ctx, opL, I.x_int, I.n_int, I.W, I.b, n, pref, A64, ld, 0, 1.0)) < 0) break;
            if (I.n_bc) {
                if ((rc = fl_prefactors(ctx, opI, I.W, n, scale, o->bc_weight, pref)) < 0) break;
                if ((rc = fl_launch_assemble_f64(ctx, opI, I.x_bc, I.n_bc, I.W, I.b, n, pref, A64, ld, I.n_int,
                                                 o->bc_weight)) < 0) break;
            }
            rc = fastlsq_lstsq(ctx, FASTLSQ_PREC_FP64, A64, FASTLSQ_F64, ld, m, n, o->mu, nullptr, 0, ld, nullptr, n,
                               nullptr, 0, 0, FASTLSQ_REFINE_CLASSICAL, 0.0, &P->factors[q], nullptr);
            if (rc < 0) break;
            double *H = P->H + h_off;
            k_sensor_matrix<<<dim3((unsigned)fl_cdiv(n, 256), (unsigned)I.n_sens), 256, 0, ctx->stream>>>(
                I.sensors, I.n_sens, I.W, I.b, n, scale, H);
            if (cudaGetLastError() != cudaSuccess) {
                rc = fl_fail(ctx, FASTLSQ_ERR_CUDA, "sensor matrix");
                break;
            }
            const fastlsq_factor *f = P->factors[q];
            InvDesc &D = P->h_desc[q];
            D.n_int = I.n_int;
            D.n_feat = n;
            D.n_sens = I.n_sens;
            D.m_aug = f->m_aug;
            D.ld = f->ld;
            D.nb = f->nb;
            D.scale = scale;
            D.x_int = I.x_int;
            D.theta = I.theta;
            D.y_obs = I.y_obs;
            D.H = H;
            D.F = (const double *)f->F;
            D.T = (const double *)f->T;
            D.beta = I.beta;
            D.loss = I.loss;
            D.dtheta = I.dtheta;
            h_off += (size_t)I.n_sens * n;
        } while (0);
    }
    if (A64) cudaFreeAsync(A64, ctx->stream);
    if (pref) cudaFreeAsync(pref, ctx->stream);
    if (rc >= 0) {
        for (const InvDesc &D : P->h_desc)
            if (D.nb > IB_NB) rc = fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_prepare: panel width %d", D.nb);
    }
    if (rc >= 0) {
        // longest first: the evaluation's work per instance grows with m_aug n
        P->h_order.resize(n_inst);
        std::iota(P->h_order.begin(), P->h_order.end(), 0);
        std::stable_sort(P->h_order.begin(), P->h_order.end(), [&](int a, int b) {
            return P->h_desc[a].m_aug * P->h_desc[a].n_feat > P->h_desc[b].m_aug * P->h_desc[b].n_feat;
        });
        e = cudaMemcpyAsync(P->d_desc, P->h_desc.data(), sizeof(InvDesc) * n_inst, cudaMemcpyHostToDevice,
                            ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(P->d_order, P->h_order.data(), sizeof(int) * n_inst, cudaMemcpyHostToDevice,
                                ctx->stream);
        // the host tables are read by the copies: finish them before returning
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) rc = fl_cuda(ctx, e, "inverse_prepare tables");
    }
    if (rc >= 0) rc = fastlsq_sync(ctx);
    if (rc < 0) {
        plan_free(P);
        return rc;
    }
    *out = P;
    return 0;
}

extern "C" int fastlsq_inverse_eval(fastlsq_ctx *ctx, const fastlsq_inverse_plan *P, int32_t threads,
                                    int32_t ctas_per_sm)
{
    if (!ctx || !P) return FASTLSQ_ERR_INVALID;
    if ((threads != 256 && threads != 512) || ctas_per_sm < 1 || ctas_per_sm > 4)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_eval: threads 256 or 512, 1..4 CTAs per SM");
    const size_t smem = ib_smem(threads, P->m_aug_max, P->n_max);
    if (smem * ctas_per_sm > (size_t)ctx->max_smem_optin)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_eval: %d CTAs per SM do not fit in shared memory",
                       ctas_per_sm);
    const int grid = std::min<int>(P->n_inst, ctx->num_sms * ctas_per_sm);
    cudaError_t e = cudaMemsetAsync(P->d_queue, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "inverse_eval queue");
    FL_PROF(ctx, FASTLSQ_K_ADJOINT);
    e = (threads == 256) ? ib_launch<256>(P, ctx->stream, grid, smem) : ib_launch<512>(P, ctx->stream, grid, smem);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "inverse_eval launch");
    return 0;
}

extern "C" int fastlsq_inverse_plan_destroy(fastlsq_inverse_plan *P)
{
    if (P) {
        cudaSetDevice(P->device);
        cudaStreamSynchronize(P->stream);
    }
    plan_free(P);
    return 0;
}

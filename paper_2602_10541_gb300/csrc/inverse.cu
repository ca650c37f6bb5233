// Batched inverse problem (Sec. 3.8 in steady form, Sec. 2.5): loss and dL/dtheta
// for many instances of uneven size, queued on one stream with no host round trip.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "qr.cuh"

int fl_launch_eval(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d, const double *W,
                   const double *b, int64_t n_feat, double scale, const double *beta, double *u);
int fl_launch_eval_adjoint(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d,
                           const double *W, const double *b, int64_t n_feat, double scale,
                           const double *g, double *grad);

namespace {

constexpr int MAX_SRC = 8;

// rhs[i] = s(x_i; theta) for i < n, 0 for n <= i < n_total (the boundary rows)
__global__ void k_gauss_dev(const double *__restrict__ x, int64_t n, const double *__restrict__ theta,
                            int n_src, double *__restrict__ out, int64_t n_total)
{
    __shared__ double th[4 * MAX_SRC];
    for (int t = threadIdx.x; t < 4 * n_src; t += blockDim.x) th[t] = theta[t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_total) return;
    double v = 0.0;
    if (i < n) {
        const double px = x[2 * i], py = x[2 * i + 1];
        for (int k = 0; k < n_src; ++k) {
            const double dx = px - th[4 * k], dy = py - th[4 * k + 1];
            v += th[4 * k + 3] * exp(-(dx * dx + dy * dy) / (2.0 * th[4 * k + 2] * th[4 * k + 2]));
        }
    }
    out[i] = v;
}

// g_s = 2 (u_s - y_s) / ns and loss = mean (u_s - y_s)^2 (one block, fixed-order sum)
__global__ void __launch_bounds__(256)
k_sensor_loss(const double *__restrict__ u, const double *__restrict__ y, int64_t ns,
              double *__restrict__ g, double *__restrict__ loss)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t s = threadIdx.x; s < ns; s += 256) {
        const double r = u[s] - y[s];
        g[s] = 2.0 * r / (double)ns;
        acc += r * r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] / (double)ns;
}

// partials [block][32] of sum_i w_i ds(x_i; theta)/dtheta, theta on the device
__global__ void __launch_bounds__(256)
k_source_grad_dev(const double *__restrict__ x, int64_t n, const double *__restrict__ theta, int n_src,
                  const double *__restrict__ w, double *__restrict__ part)
{
    __shared__ double th[4 * MAX_SRC];
    __shared__ double red[256];
    for (int t = threadIdx.x; t < 4 * n_src; t += blockDim.x) th[t] = theta[t];
    __syncthreads();
    double acc[4 * MAX_SRC];
    for (int q = 0; q < 4 * n_src; ++q) acc[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double px = x[2 * i], py = x[2 * i + 1], wi = w[i];
        for (int k = 0; k < n_src; ++k) {
            const double *t = th + 4 * k;
            const double dx = px - t[0], dy = py - t[1];
            const double r2 = dx * dx + dy * dy, w2 = t[2] * t[2];
            const double e = exp(-r2 / (2.0 * w2));
            acc[4 * k + 0] += wi * t[3] * e * dx / w2;
            acc[4 * k + 1] += wi * t[3] * e * dy / w2;
            acc[4 * k + 2] += wi * t[3] * e * r2 / (w2 * t[2]);
            acc[4 * k + 3] += wi * e;
        }
    }
    for (int q = 0; q < 4 * n_src; ++q) {
        red[threadIdx.x] = acc[q];
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 32 + q] = red[0];
        __syncthreads();
    }
}

__global__ void k_sum_blocks(const double *__restrict__ part, int nblk, int nq, double *__restrict__ out)
{
    const int q = threadIdx.x;
    if (q >= nq) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[b * 32 + q];
    out[q] = s;
}

}  // namespace

int fl_matvec64(fastlsq_ctx *ctx, const double *A, int64_t ld, int64_t m, int64_t n,
                const double *v, double *out);

extern "C" int fastlsq_inverse_batch(fastlsq_ctx *ctx, const fastlsq_inverse_instance *inst,
                                     int32_t n_inst, const fastlsq_op *op, int32_t n_src,
                                     const fastlsq_inverse_opts *o)
{
    if (!ctx || !inst || !op || !o || n_inst < 0) return FASTLSQ_ERR_INVALID;
    if (n_src < 1 || n_src > MAX_SRC) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse: n_src 1..%d", MAX_SRC);
    if (o->prec != FASTLSQ_PREC_FP64 && o->prec != FASTLSQ_PREC_MIXED)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse: precision");
    fl_op_params opL;
    FL_TRY(fl_pack_op(ctx, op, &opL));
    if (opL.d != 2 || opL.n_pp != 0) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse: 2-D operator without per-point terms");
    fl_op_params opI;
    memset(&opI, 0, sizeof(opI));
    opI.d = 2;
    opI.n_terms = 1;
    opI.coef[0] = 1.0;
    int64_t m_max = 0, n_max = 0, ns_max = 0;
    for (int q = 0; q < n_inst; ++q) {
        const fastlsq_inverse_instance &I = inst[q];
        if (I.n_int < 1 || I.n_bc < 0 || I.n_feat < 1 || I.n_feat > FL_MAX_FEAT || I.n_sens < 1 ||
            !I.x_int || (I.n_bc && !I.x_bc) || !I.W || !I.b || !I.sensors || !I.y_obs || !I.theta ||
            !I.beta || !I.loss || !I.dtheta)
            return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse: bad instance %d", q);
        m_max = std::max<int64_t>(m_max, fl_round_up(I.n_int + I.n_bc, 4));
        n_max = std::max<int64_t>(n_max, I.n_feat);
        ns_max = std::max<int64_t>(ns_max, I.n_sens);
    }
    if (n_inst == 0) return 0;
    const bool mixed = o->prec == FASTLSQ_PREC_MIXED;
    // pooled buffers sized for the largest instance (stream-ordered allocations)
    const int nblk_g = 64;
    size_t bytes64 = sizeof(double) * (m_max * n_max + 2 * m_max + 3 * n_max + 2 * ns_max + 32 * nblk_g + 64);
    double *pool64 = nullptr;
    float *A32 = nullptr;
    double *pref = nullptr;
    cudaError_t e = cudaMallocAsync(&pool64, bytes64, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&pref, sizeof(double) * (2 + FL_MAX_PP) * n_max, ctx->stream);
    if (e == cudaSuccess && mixed) e = cudaMallocAsync(&A32, sizeof(float) * m_max * n_max, ctx->stream);
    if (e != cudaSuccess) {
        if (pool64) cudaFreeAsync(pool64, ctx->stream);
        if (pref) cudaFreeAsync(pref, ctx->stream);
        return fl_cuda(ctx, e, "inverse batch buffers");
    }
    double *A64 = pool64;
    double *rhs = A64 + m_max * n_max;
    double *grad_rhs = rhs + m_max;
    double *gbeta = grad_rhs + m_max;
    double *v = gbeta + n_max;
    double *u_s = v + n_max + n_max;
    double *g = u_s + ns_max;
    double *part = g + ns_max;
    int rc = 0;
    for (int q = 0; q < n_inst && rc >= 0; ++q) {
        const fastlsq_inverse_instance &I = inst[q];
        const int64_t n = I.n_feat, m = I.n_int + I.n_bc, ld = fl_round_up(m, 4);
        const double scale = 1.0 / sqrt((double)n);
        fastlsq_factor *fac = nullptr;
        do {
            // operator rows: interior -L, boundary lambda * identity (FP64, and FP32 for MIXED)
            if ((rc = fl_prefactors(ctx, opL, I.W, n, scale, 1.0, pref)) < 0) break;
            if ((rc = fl_launch_assemble_f64(ctx, opL, I.x_int, I.n_int, I.W, I.b, n, pref, A64, ld, 0, 1.0)) < 0) break;
            if (mixed && (rc = fl_launch_assemble_f32(ctx, opL, I.x_int, I.n_int, I.W, I.b, n, pref, A32, ld, 0, 1.0)) < 0) break;
            if (I.n_bc) {
                if ((rc = fl_prefactors(ctx, opI, I.W, n, scale, o->bc_weight, pref)) < 0) break;
                if ((rc = fl_launch_assemble_f64(ctx, opI, I.x_bc, I.n_bc, I.W, I.b, n, pref, A64, ld, I.n_int,
                                                 o->bc_weight)) < 0) break;
                if (mixed && (rc = fl_launch_assemble_f32(ctx, opI, I.x_bc, I.n_bc, I.W, I.b, n, pref, A32, ld,
                                                          I.n_int, o->bc_weight)) < 0) break;
            }
            {
                FL_PROF(ctx, FASTLSQ_K_RHS);
                k_gauss_dev<<<(unsigned)fl_cdiv(ld, 256), 256, 0, ctx->stream>>>(I.x_int, I.n_int, I.theta, n_src,
                                                                                 rhs, ld);
            }
            // forward: factor (kept for the adjoint) and solve
            rc = fastlsq_lstsq(ctx, (fastlsq_prec)o->prec, mixed ? (const void *)A32 : (const void *)A64,
                               mixed ? FASTLSQ_F32 : FASTLSQ_F64, ld, m, n, o->mu, rhs, 1, ld, I.beta, n, A64,
                               ld, mixed ? o->refine_iters : 0, FASTLSQ_REFINE_CGLS, o->refine_tol, &fac,
                               nullptr);
            if (rc < 0) break;
            // sensors, loss and dL/du_s
            if ((rc = fl_launch_eval(ctx, I.sensors, I.n_sens, 2, I.W, I.b, n, scale, I.beta, u_s)) < 0) break;
            {
                FL_PROF(ctx, FASTLSQ_K_ADJOINT);
                k_sensor_loss<<<1, 256, 0, ctx->stream>>>(u_s, I.y_obs, I.n_sens, g, I.loss);
            }
            // adjoint: grad_beta = H_s^T g ; v ; grad_rhs = A v ; dL/dtheta
            if ((rc = fl_launch_eval_adjoint(ctx, I.sensors, I.n_sens, 2, I.W, I.b, n, scale, g, gbeta)) < 0) break;
            rc = fastlsq_backward(ctx, fac, gbeta, v, grad_rhs, A64, ld, mixed ? o->adjoint_iters : 0,
                                  o->adjoint_tol);
            if (rc < 0) break;
            {
                FL_PROF_N(ctx, FASTLSQ_K_ADJOINT, 2);
                k_source_grad_dev<<<nblk_g, 256, 0, ctx->stream>>>(I.x_int, I.n_int, I.theta, n_src, grad_rhs,
                                                                   part);
                k_sum_blocks<<<1, 32, 0, ctx->stream>>>(part, nblk_g, 4 * n_src, I.dtheta);
            }
            if (cudaGetLastError() != cudaSuccess) rc = fl_fail(ctx, FASTLSQ_ERR_CUDA, "inverse batch kernels");
        } while (0);
        if (fac) fastlsq_factor_destroy(fac);
    }
    cudaFreeAsync(pool64, ctx->stream);
    cudaFreeAsync(pref, ctx->stream);
    if (A32) cudaFreeAsync(A32, ctx->stream);
    return rc < 0 ? rc : 0;
}

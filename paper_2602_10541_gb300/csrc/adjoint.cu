// Adjoint pieces of the differentiable solve (Sec. 2.5; Sec. 3.8): the FP64
// product A v, and the on-the-fly contraction that gives gradients with respect
// to operator coefficients,
//   dL/dc_t = sum_ij (r_i v_j - (A v)_i beta_j) * s * D^{alpha_t} phi_j(x_i),
// which follows from differentiating (A^T A + mu I) beta = A^T rhs.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int MV_ROWS = 256;
constexpr int MV_COLS = 128;

__global__ void __launch_bounds__(MV_ROWS)
k_matvec_partial(const double *__restrict__ A, int64_t ld, int64_t m, int64_t n,
                 const double *__restrict__ v, double *__restrict__ part)
{
    __shared__ double sv[MV_COLS];
    const int64_t j0 = (int64_t)blockIdx.y * MV_COLS;
    const int nc = (int)fl_min64(MV_COLS, n - j0);
    for (int t = threadIdx.x; t < nc; t += blockDim.x) sv[t] = v[j0 + t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * MV_ROWS + threadIdx.x;
    if (i >= m) return;
    double acc = 0.0;
    const double *a = A + i + j0 * ld;
#pragma unroll 8
    for (int c = 0; c < nc; ++c) acc = fma(a[(int64_t)c * ld], sv[c], acc);
    part[(int64_t)blockIdx.y * m + i] = acc;
}

__global__ void k_matvec_reduce(const double *__restrict__ part, int nsplit, int64_t m,
                                double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * m + i];
    out[i] = s;
}

constexpr int CG_THREADS = 128;
constexpr int CG_COLS = 256;

// per block: partial sums of every term over its rows x column chunk
__global__ void __launch_bounds__(CG_THREADS)
k_coef_grad(const double *__restrict__ x, int64_t n_rows, fl_op_params op,
            const double *__restrict__ W, const double *__restrict__ b, int64_t n_feat,
            double scale, const double *__restrict__ r, const double *__restrict__ Av,
            const double *__restrict__ v, const double *__restrict__ beta,
            double *__restrict__ part)
{
    __shared__ double red[CG_THREADS];
    const int64_t i = (int64_t)blockIdx.x * CG_THREADS + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * CG_COLS;
    const int64_t j1 = fl_min64(n_feat, j0 + CG_COLS);
    double acc[FL_MAX_TERMS];
    for (int t = 0; t < op.n_terms; ++t) acc[t] = 0.0;
    if (i < n_rows) {
        const double ri = r[i], avi = Av[i];
        for (int64_t j = j0; j < j1; ++j) {
            double z = b[j];
            for (int k = 0; k < op.d; ++k) z = fma(W[j * op.d + k], x[i * op.d + k], z);
            double sn, cs;
            sincos(z, &sn, &cs);
            const double wgt = ri * v[j] - avi * beta[j];
            for (int t = 0; t < op.n_terms; ++t) {
                double mlt = 1.0;
                int order = 0;
                for (int k = 0; k < op.d; ++k)
                    for (int q = 0; q < op.alpha[t][k]; ++q) {
                        mlt *= W[j * op.d + k];
                        ++order;
                    }
                double phi = (order & 1) ? cs : sn;
                if ((order >> 1) & 1) phi = -phi;
                acc[t] = fma(mlt * phi, wgt, acc[t]);
            }
        }
    }
    for (int t = 0; t < op.n_terms; ++t) {
        red[threadIdx.x] = acc[t];
        __syncthreads();
        for (int s = CG_THREADS / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            part[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * FL_MAX_TERMS + t] = scale * red[0];
        __syncthreads();
    }
}

// out[q] = sum over blocks, in block order, of part[blk * stride + q] (q < ncols)
__global__ void k_sum_blocks(const double *__restrict__ part, int64_t nblk, int stride, int ncols,
                             double *__restrict__ out)
{
    const int q = threadIdx.x;
    if (q >= ncols) return;
    double acc = 0.0;
    for (int64_t blk = 0; blk < nblk; ++blk) acc += part[blk * stride + q];
    out[q] = acc;
}

}  // namespace

int fl_reduce_blocks_to_host(fastlsq_ctx *ctx, double *part, int64_t nblk, int stride, int ncols,
                             double *host_out)
{
    // the sums land in the row after the last block's partials (the caller sizes part
    // for nblk + 1 rows), then one copy of ncols values to the host
    double *sums = part + nblk * stride;
    {
    FL_PROF(ctx, FASTLSQ_K_ADJOINT);
    k_sum_blocks<<<1, 64, 0, ctx->stream>>>(part, nblk, stride, ncols, sums);
    FL_CHECK_LAUNCH(ctx, "sum_blocks");
    }
    cudaError_t e = cudaMemcpyAsync(host_out, sums, sizeof(double) * ncols, cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "gradient readback");
    return 0;
}

int fl_matvec64(fastlsq_ctx *ctx, const double *A, int64_t ld, int64_t m, int64_t n,
                const double *v, double *out)
{
    if (m == 0) return 0;
    int nsplit = (int)fl_cdiv(n, MV_COLS);
    double *part = (double *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(double) * nsplit * m);
    if (!part) return FASTLSQ_ERR_NOMEM;
    FL_PROF_N(ctx, FASTLSQ_K_RESIDUAL, 2);
    k_matvec_partial<<<dim3((unsigned)fl_cdiv(m, MV_ROWS), (unsigned)nsplit), MV_ROWS, 0,
                       ctx->stream>>>(A, ld, m, n, v, part);
    FL_CHECK_LAUNCH(ctx, "matvec_partial");
    k_matvec_reduce<<<(unsigned)fl_cdiv(m, 256), 256, 0, ctx->stream>>>(part, nsplit, m, out);
    FL_CHECK_LAUNCH(ctx, "matvec_reduce");
    return 0;
}

int fl_launch_coef_grad(fastlsq_ctx *ctx, const double *x, int64_t n_rows, const fl_op_params &op,
                        const double *W, const double *b, int64_t n_feat, double scale,
                        const double *r, const double *Av, const double *v, const double *beta,
                        double *grad_host)
{
    for (int t = 0; t < op.n_terms; ++t) grad_host[t] = 0.0;
    if (n_rows == 0 || op.n_terms == 0) return 0;
    dim3 grid((unsigned)fl_cdiv(n_rows, CG_THREADS), (unsigned)fl_cdiv(n_feat, CG_COLS));
    size_t nblk = (size_t)grid.x * grid.y;
    double *part = (double *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(double) * (nblk + 1) * FL_MAX_TERMS);
    if (!part) return FASTLSQ_ERR_NOMEM;
    {
    FL_PROF(ctx, FASTLSQ_K_ADJOINT);
    k_coef_grad<<<grid, CG_THREADS, 0, ctx->stream>>>(x, n_rows, op, W, b, n_feat, scale, r, Av, v,
                                                      beta, part);
    FL_CHECK_LAUNCH(ctx, "coef_grad");
    }
    return fl_reduce_blocks_to_host(ctx, part, (int64_t)nblk, FL_MAX_TERMS, op.n_terms, grad_host);
}

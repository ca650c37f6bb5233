// Learnable bandwidth (App. "Learnable Bandwidth via Reparameterisation", Alg. 2):
// gradients of a loss with respect to the feature weights W and biases b through the
// exact inner solve, and their contraction with the frozen base weights W_hat
// (W = sigma W_hat, eq. reparam_scalar; W_j = L W_hat_j, eq. reparam_cholesky).
//
// For a block A_ij = rw * s * sum_t c_t D^{alpha_t} phi_j(x_i) = P_j sin z_ij + Q_j cos z_ij
// (eq. cyclic, P and Q the column prefactors) the derivatives are
//   dA_ij/dW_jk = Pk_j sin z + Qk_j cos z + x_ik (P_j cos z - Q_j sin z),
//   dA_ij/db_j  = P_j cos z - Q_j sin z,
// with Pk, Qk the prefactors' derivatives in W_jk.  The loss weights of the adjoint
// bilinear form are w_ij = r_i (c_v v_j + c_rb beta_j) + c_av (A v)_i beta_j, so
//   sum_i w_ij dA_ij/dW_jk = v1_j [Pk S_r + Qk C_r + P Xc_r,k - Q Xs_r,k]
//                          + v2_j [Pk S_a + Qk C_a + P Xc_a,k - Q Xs_a,k]
// with v1 = c_v v + c_rb beta, v2 = c_av beta and the row sums S_r = sum_i r_i sin z,
// C_r = sum_i r_i cos z, Xs_r,k = sum_i r_i x_ik sin z, Xc_r,k likewise, and the same
// with Av in place of r.  One pass over the rows (thread per column, FP64 sincos on
// the fly, nothing stored) accumulates the row sums per row chunk; a second kernel
// adds the chunks in order and applies the prefactors.
#include <cmath>

#include "common.cuh"

namespace {

constexpr int WG_THREADS = 128;   // columns per CTA, one per thread
constexpr int WG_ROWS = 128;      // rows per chunk (one CTA row of the grid)

template <int D, bool AV>
__global__ void __launch_bounds__(WG_THREADS)
k_wgrad_partial(const double *__restrict__ x, int64_t n_rows, const double *__restrict__ W,
                const double *__restrict__ b, int64_t n_feat, const double *__restrict__ r,
                const double *__restrict__ Av, double *__restrict__ part)
{
    constexpr int H = 2 + 2 * D;               // sums per weight vector
    constexpr int NS = AV ? 2 * H : H;
    __shared__ double sx[WG_ROWS * D];
    __shared__ double sr[WG_ROWS];
    __shared__ double sa[AV ? WG_ROWS : 1];
    const int64_t i0 = (int64_t)blockIdx.y * WG_ROWS;
    const int nr = (int)fl_min64(WG_ROWS, n_rows - i0);
    for (int t = threadIdx.x; t < nr * D; t += WG_THREADS) sx[t] = x[i0 * D + t];
    for (int t = threadIdx.x; t < nr; t += WG_THREADS) {
        sr[t] = r[i0 + t];
        if constexpr (AV) sa[t] = Av[i0 + t];
    }
    __syncthreads();
    const int64_t j = (int64_t)blockIdx.x * WG_THREADS + threadIdx.x;
    if (j >= n_feat) return;
    double w[D];
#pragma unroll
    for (int k = 0; k < D; ++k) w[k] = W[j * D + k];
    const double bj = b[j];
    double acc[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) acc[q] = 0.0;
    for (int i = 0; i < nr; ++i) {
        double z = bj;
#pragma unroll
        for (int k = 0; k < D; ++k) z = fma(w[k], sx[i * D + k], z);
        double sn, cs;
        sincos(z, &sn, &cs);
        const double rs = sr[i] * sn, rc = sr[i] * cs;
        acc[0] += rs;
        acc[1] += rc;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            acc[2 + 2 * k] = fma(rs, sx[i * D + k], acc[2 + 2 * k]);
            acc[3 + 2 * k] = fma(rc, sx[i * D + k], acc[3 + 2 * k]);
        }
        if constexpr (AV) {
            const double as = sa[i] * sn, ac = sa[i] * cs;
            acc[H] += as;
            acc[H + 1] += ac;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                acc[H + 2 + 2 * k] = fma(as, sx[i * D + k], acc[H + 2 + 2 * k]);
                acc[H + 3 + 2 * k] = fma(ac, sx[i * D + k], acc[H + 3 + 2 * k]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) part[((int64_t)blockIdx.y * NS + q) * n_feat + j] = acc[q];
}

// adds the row chunks in chunk order and applies the column prefactors (accumulates)
template <int D, bool AV>
__global__ void k_wgrad_final(const double *__restrict__ part, int nchunk, fl_op_params op,
                              double ws, const double *__restrict__ W,
                              const double *__restrict__ beta, const double *__restrict__ v,
                              double c_v, double c_rb, double c_av, int64_t n_feat,
                              double *__restrict__ gW, double *__restrict__ gb)
{
    constexpr int H = 2 + 2 * D;
    constexpr int NS = AV ? 2 * H : H;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_feat) return;
    double s[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) s[q] = 0.0;
    for (int c = 0; c < nchunk; ++c)
#pragma unroll
        for (int q = 0; q < NS; ++q) s[q] += part[((int64_t)c * NS + q) * n_feat + j];
    double w[D];
#pragma unroll
    for (int k = 0; k < D; ++k) w[k] = W[j * D + k];
    // prefactors of the block and their derivatives in W_jk, grouped by the phase
    // Phi_{|alpha| mod 4}: sin (+P), cos (+Q), -sin (-P), -cos (-Q)
    double P = 0.0, Q = 0.0, Pk[D], Qk[D];
#pragma unroll
    for (int k = 0; k < D; ++k) Pk[k] = Qk[k] = 0.0;
    for (int t = 0; t < op.n_terms; ++t) {
        int ord = 0;
        double m = ws * op.coef[t];
        for (int k = 0; k < D; ++k)
            for (int q = 0; q < op.alpha[t][k]; ++q) {
                m *= w[k];
                ++ord;
            }
        const double sg = ((ord >> 1) & 1) ? -1.0 : 1.0;
        if (ord & 1) Q += sg * m;
        else P += sg * m;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (op.alpha[t][k] == 0) continue;
            double dm = ws * op.coef[t] * (double)op.alpha[t][k];
            for (int l = 0; l < D; ++l) {
                const int p = (l == k) ? op.alpha[t][l] - 1 : op.alpha[t][l];
                for (int q = 0; q < p; ++q) dm *= w[l];
            }
            if (ord & 1) Qk[k] += sg * dm;
            else Pk[k] += sg * dm;
        }
    }
    const double v1 = (v ? c_v * v[j] : 0.0) + c_rb * beta[j];
    const double v2 = c_av * beta[j];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        double g = v1 * (Pk[k] * s[0] + Qk[k] * s[1] + P * s[3 + 2 * k] - Q * s[2 + 2 * k]);
        if constexpr (AV)
            g += v2 * (Pk[k] * s[H] + Qk[k] * s[H + 1] + P * s[H + 3 + 2 * k] - Q * s[H + 2 + 2 * k]);
        gW[j * D + k] += g;
    }
    if (gb) {
        double g = v1 * (P * s[1] - Q * s[0]);
        if constexpr (AV) g += v2 * (P * s[H + 1] - Q * s[H]);
        gb[j] += g;
    }
}

// out[a*d + c] = sum_j gW[j][a] W_hat[j][c], one CTA per (a, c), fixed-order reduction
__global__ void __launch_bounds__(256)
k_bw_contract(const double *__restrict__ gW, const double *__restrict__ What, int64_t n_feat,
              int d, double *__restrict__ out)
{
    __shared__ double red[256];
    const int a = blockIdx.x / d, c = blockIdx.x % d;
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < n_feat; j += 256) acc = fma(gW[j * d + a], What[j * d + c], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// out[d*d] = trace: dL/dsigma for W = sigma W_hat
__global__ void k_bw_trace(double *__restrict__ out, int d)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int a = 0; a < d; ++a) t += out[a * d + a];
        out[d * d] = t;
    }
}

__global__ void k_rsub(const double *__restrict__ rhs, int64_t m, double *__restrict__ r)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) r[i] = rhs[i] - r[i];
}

template <int D>
int launch_wgrad(fastlsq_ctx *ctx, const double *x, int64_t n_rows, const fl_op_params &op,
                 double ws, const double *W, const double *b, int64_t n_feat, const double *r,
                 const double *beta, const double *v, const double *Av, double c_v, double c_rb,
                 double c_av, double *gW, double *gb)
{
    const int nchunk = (int)fl_cdiv(n_rows, WG_ROWS);
    const int ns = (2 + 2 * D) * (Av ? 2 : 1);
    double *part = (double *)fl_ws(ctx, FL_WS_WGRAD, sizeof(double) * (size_t)nchunk * ns * n_feat);
    if (!part) return FASTLSQ_ERR_NOMEM;
    const dim3 grid((unsigned)fl_cdiv(n_feat, WG_THREADS), (unsigned)nchunk);
    const unsigned fb = (unsigned)fl_cdiv(n_feat, 128);
    FL_PROF_N(ctx, FASTLSQ_K_ADJOINT, 2);
    if (Av) {
        k_wgrad_partial<D, true><<<grid, WG_THREADS, 0, ctx->stream>>>(x, n_rows, W, b, n_feat, r, Av, part);
        k_wgrad_final<D, true><<<fb, 128, 0, ctx->stream>>>(part, nchunk, op, ws, W, beta, v, c_v, c_rb,
                                                            c_av, n_feat, gW, gb);
    } else {
        k_wgrad_partial<D, false><<<grid, WG_THREADS, 0, ctx->stream>>>(x, n_rows, W, b, n_feat, r, Av, part);
        k_wgrad_final<D, false><<<fb, 128, 0, ctx->stream>>>(part, nchunk, op, ws, W, beta, v, c_v, c_rb,
                                                             c_av, n_feat, gW, gb);
    }
    FL_CHECK_LAUNCH(ctx, "weight_grad");
    return 0;
}

}  // namespace

int fl_matvec64(fastlsq_ctx *ctx, const double *A, int64_t ld, int64_t m, int64_t n,
                const double *v, double *out);

extern "C" int fastlsq_weight_grad(fastlsq_ctx *ctx, const double *x, int64_t n_rows,
                                   const fastlsq_op *op, double row_weight, const double *W,
                                   const double *b, int64_t n_feat, double scale, const double *r,
                                   const double *beta, const double *v, const double *Av,
                                   double c_v, double c_rb, double c_av, double *gW, double *gb)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    fl_op_params p;
    FL_TRY(fl_pack_op(ctx, op, &p));
    if (p.n_pp != 0) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "weight_grad: per-point terms");
    if (n_rows < 0 || n_feat < 1 || !W || !b || !beta || !gW || (n_rows > 0 && (!x || !r)))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "weight_grad: bad arguments");
    if (n_rows == 0) return 0;
    const double ws = row_weight * scale;
    switch (p.d) {
#define FL_WG(DD) \
    case DD: return launch_wgrad<DD>(ctx, x, n_rows, p, ws, W, b, n_feat, r, beta, v, Av, c_v, c_rb, c_av, gW, gb);
        FL_WG(1) FL_WG(2) FL_WG(3) FL_WG(4) FL_WG(5) FL_WG(6) FL_WG(7) FL_WG(8)
#undef FL_WG
    default: return fl_fail(ctx, FASTLSQ_ERR_INVALID, "weight_grad: dimension %d", p.d);
    }
}

extern "C" int fastlsq_bandwidth_grad(fastlsq_ctx *ctx, const double *gW, const double *W_hat,
                                      int64_t n_feat, int32_t d, double *out)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (!gW || !W_hat || !out || n_feat < 1 || d < 1 || d > FL_MAX_D)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "bandwidth_grad: bad arguments");
    FL_PROF_N(ctx, FASTLSQ_K_ADJOINT, 2);
    k_bw_contract<<<d * d, 256, 0, ctx->stream>>>(gW, W_hat, n_feat, d, out);
    k_bw_trace<<<1, 32, 0, ctx->stream>>>(out, d);
    FL_CHECK_LAUNCH(ctx, "bandwidth_grad");
    return 0;
}

extern "C" int fastlsq_residual(fastlsq_ctx *ctx, const double *A, int64_t ld, int64_t m,
                                int64_t n, const double *beta, const double *rhs, double *r)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (m < 0 || n < 1 || ld < m || (m > 0 && (!A || !beta || !rhs || !r)))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "residual: bad arguments");
    if (m == 0) return 0;
    FL_TRY(fl_matvec64(ctx, A, ld, m, n, beta, r));
    FL_PROF(ctx, FASTLSQ_K_VECTOR);
    k_rsub<<<(unsigned)fl_cdiv(m, 256), 256, 0, ctx->stream>>>(rhs, m, r);
    FL_CHECK_LAUNCH(ctx, "residual");
    return 0;
}

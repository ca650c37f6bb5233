// Operator assembly (Sec. 2.2 eq. cyclic; Sec. 2.3 eq. linear_system; Alg. 1
// steps 3-4), feature evaluation at points (eq. approximation) and the
// right-hand sides of the manufactured problems.
//
// Column prefactors.  For term t with multi-index alpha_t, the entry is
//   coef_t * s * (prod_k W_jk^alpha_tk) * Phi_{|alpha_t| mod 4}(z),
// and Phi_{0,1,2,3} = (sin, cos, -sin, -cos).  Summing the constant-coefficient
// terms by the parity of |alpha_t| folds the whole operator into two numbers per
// column:  A_ij = P_j sin z_ij + Q_j cos z_ij  (times the row weight), with
//   P_j = s sum_{|alpha| even} coef_t m_tj (-1)^{|alpha|/2},
//   Q_j = s sum_{|alpha| odd}  coef_t m_tj (-1)^{(|alpha|-1)/2}.
// Per-point terms (the Newton Jacobian's N'(u_i) phi_j) keep their own column
// multiplier M_qj = s m_qj (+-1) and a per-row coefficient.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "common.cuh"

namespace {

__global__ void k_prefactors(fl_op_params op, const double *__restrict__ W, int64_t n_feat,
                             double scale_rw, double *__restrict__ pref)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n_feat) return;
    double w[FL_MAX_D];
#pragma unroll
    for (int k = 0; k < FL_MAX_D; ++k) w[k] = (k < op.d) ? W[j * op.d + k] : 0.0;
    double P = 0.0, Q = 0.0;
    for (int t = 0; t < op.n_terms; ++t) {
        double m = 1.0;
        int order = 0;
        for (int k = 0; k < op.d; ++k)
            for (int r = 0; r < op.alpha[t][k]; ++r) {
                m *= w[k];
                ++order;
            }
        double sgn = ((order >> 1) & 1) ? -1.0 : 1.0;   // Phi_2, Phi_3 carry a minus sign
        if (order & 1) Q += op.coef[t] * m * sgn;
        else P += op.coef[t] * m * sgn;
    }
    pref[j] = scale_rw * P;
    pref[n_feat + j] = scale_rw * Q;
    for (int q = 0; q < op.n_pp; ++q) {
        double m = 1.0;
        int order = 0;
        for (int k = 0; k < op.d; ++k)
            for (int r = 0; r < op.pp_alpha[q][k]; ++r) {
                m *= w[k];
                ++order;
            }
        double sgn = ((order >> 1) & 1) ? -1.0 : 1.0;
        pref[(2 + q) * n_feat + j] = scale_rw * m * sgn;
    }
}

constexpr int ASM_ROWS = 128;   // rows per CTA (32 lanes x 4 rows)
constexpr int ASM_COLS = 64;    // columns per CTA (8 warps x 8 columns)
constexpr int ASM_THREADS = 256;

struct fl_pp_rows {
    const double *c[FL_MAX_PP];
};

// FP32 assembly: z in float FMAs, Cody-Waite reduction to [-pi, pi] with a
// three-part 2 pi, SFU sin/cos, float4 stores of 4 consecutive rows.  The point
// dimension D is a template parameter, so the inner loop holds exactly D FMAs.
// CTA tile: 128 rows (32 lanes x 4 rows) x 256 columns; the column data (W, b, P,
// Q) are converted to float once per CTA into shared memory, the thread's 4 points
// once per thread into registers.  NPP is the number of per-point terms compiled in:
// 0 for plain operators (no registers or shared memory spent on them), FL_MAX_PP for
// operators with per-point coefficients (Newton Jacobians, variable coefficients).
constexpr int AF_ROWS = 128;
constexpr int AF_COLS = 256;
constexpr int AF_THREADS = 256;

template <int D, bool NEED_COS, int NPP>
__global__ void __launch_bounds__(AF_THREADS)
k_assemble_f32(const double *__restrict__ x, int64_t n_rows,
               const double *__restrict__ W, const double *__restrict__ b, int64_t n_feat,
               const double *__restrict__ pref, int n_pp, unsigned pp_cos_mask, fl_pp_rows pp,
               float *__restrict__ A, int64_t ldA, int64_t row_offset,
               float c1, float c2, float c3)
{
    __shared__ float sW[D][AF_COLS];
    __shared__ float sB[AF_COLS], sP[AF_COLS], sQ[NEED_COS ? AF_COLS : 1];
    __shared__ float sM[NPP > 0 ? NPP : 1][AF_COLS];
    __shared__ float sX[AF_ROWS][D];                     // the CTA's points, converted once

    const int64_t col0 = (int64_t)blockIdx.y * AF_COLS;
    const int64_t row0 = (int64_t)blockIdx.x * AF_ROWS;
    const int ncol = (int)fl_min64(AF_COLS, n_feat - col0);
    for (int t = threadIdx.x; t < ncol * D; t += AF_THREADS) {
        const int c = t / D, k = t % D;                  // consecutive threads: consecutive W
        sW[k][c] = (float)W[(col0 + c) * D + k];
    }
    for (int t = threadIdx.x; t < ncol; t += AF_THREADS) {
        sB[t] = (float)b[col0 + t];
        sP[t] = (float)pref[col0 + t];
        if (NEED_COS) sQ[t] = (float)pref[n_feat + col0 + t];
        if constexpr (NPP > 0)
            for (int q = 0; q < n_pp; ++q) sM[q][t] = (float)pref[(2 + q) * n_feat + col0 + t];
    }

    for (int t = threadIdx.x; t < AF_ROWS * D; t += AF_THREADS) {
        const int64_t i = row0 + t / D;
        sX[t / D][t % D] = (i < n_rows) ? (float)x[row0 * D + t] : 0.f;   // consecutive reads
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t r0 = row0 + 4 * lane;
    float xr[4][D];
    float cpt[NPP > 0 ? NPP : 1][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = r0 + u;
        const bool ok = i < n_rows;
#pragma unroll
        for (int k = 0; k < D; ++k) xr[u][k] = sX[4 * lane + u][k];
#pragma unroll
        for (int q = 0; q < NPP; ++q) cpt[q][u] = (ok && q < n_pp) ? (float)pp.c[q][i] : 0.f;
    }
    const bool full = (r0 + 3 < n_rows);
    const int64_t gr = row_offset + r0;
    const bool vec = full && ((gr & 3) == 0) && ((ldA & 3) == 0) &&
                     ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    const float inv2pi = 0.159154943091895335768883763372514362f;

#pragma unroll 4
    for (int c = warp; c < ncol; c += AF_THREADS / 32) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float z = sB[c];
#pragma unroll
            for (int k = 0; k < D; ++k) z = fmaf(sW[k][c], xr[u][k], z);
            const float qn = rintf(z * inv2pi);
            float r = fmaf(-qn, c1, z);
            r = fmaf(-qn, c2, r);
            r = fmaf(-qn, c3, r);
            const float sn = __sinf(r);
            float val = sP[c] * sn;
            float cs = 0.f;
            if (NEED_COS) {
                cs = __cosf(r);
                val = fmaf(sQ[c], cs, val);
            }
            if constexpr (NPP > 0) {                      // per-point terms
#pragma unroll
                for (int q = 0; q < NPP; ++q) {
                    if (q >= n_pp) break;
                    const float phi = ((pp_cos_mask >> q) & 1) ? (NEED_COS ? cs : __cosf(r)) : sn;
                    val = fmaf(cpt[q][u] * sM[q][c], phi, val);
                }
            }
            v[u] = val;
        }
        float *dst = A + (col0 + c) * ldA + gr;
        if (vec) {
            *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (r0 + u < n_rows) dst[u] = v[u];
        }
    }
}

// FP64 assembly: double FMAs and double-precision sin/cos (CUDA's sin, cos).  Tiles of
// ASM_ROWS x ASM_COLS entries, tile t at row block t % row blocks and column block
// t / row blocks; a CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... (one tile
// per CTA when the grid covers them all, else a persistent grid whose small footprint
// leaves the SMs' other warp slots to kernels of other streams: the kernel is bound by
// the FP64 pipe, which the FP32 and tensor-core kernels beside it do not use).
template <bool NEED_COS, int NPP>
__global__ void __launch_bounds__(ASM_THREADS)
k_assemble_f64(const double *__restrict__ x, int64_t n_rows, int d,
               const double *__restrict__ W, const double *__restrict__ b, int64_t n_feat,
               const double *__restrict__ pref, int n_pp, unsigned pp_cos_mask, fl_pp_rows pp,
               double *__restrict__ A, int64_t ldA, int64_t row_offset)
{
    __shared__ double sW[ASM_COLS][FL_MAX_D];
    __shared__ double sB[ASM_COLS], sP[ASM_COLS], sQ[ASM_COLS];
    __shared__ double sM[NPP > 0 ? NPP : 1][ASM_COLS];
    const int64_t nrb = (n_rows + ASM_ROWS - 1) / ASM_ROWS;
    const int64_t ntiles = nrb * ((n_feat + ASM_COLS - 1) / ASM_COLS);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t col0 = (tile / nrb) * ASM_COLS;
        const int64_t row0 = (tile % nrb) * ASM_ROWS;
        __syncthreads();                        // the previous tile's reads of the staging
        for (int t = threadIdx.x; t < ASM_COLS; t += blockDim.x) {
            int64_t j = col0 + t;
            bool ok = j < n_feat;
            for (int k = 0; k < FL_MAX_D; ++k) sW[t][k] = (ok && k < d) ? W[j * d + k] : 0.0;
            sB[t] = ok ? b[j] : 0.0;
            sP[t] = ok ? pref[j] : 0.0;
            sQ[t] = ok ? pref[n_feat + j] : 0.0;
            if constexpr (NPP > 0)
                for (int q = 0; q < n_pp; ++q) sM[q][t] = ok ? pref[(2 + q) * n_feat + j] : 0.0;
        }
        __syncthreads();
        double xr[4][FL_MAX_D];
        double cpt[NPP > 0 ? NPP : 1][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int64_t i = row0 + lane + 32 * u;
            bool ok = i < n_rows;
#pragma unroll
            for (int k = 0; k < FL_MAX_D; ++k) xr[u][k] = (ok && k < d) ? x[i * d + k] : 0.0;
#pragma unroll
            for (int q = 0; q < NPP; ++q) cpt[q][u] = (ok && q < n_pp) ? pp.c[q][i] : 0.0;
        }
        for (int cc = 0; cc < ASM_COLS / 8; ++cc) {
            const int c = warp * (ASM_COLS / 8) + cc;
            const int64_t j = col0 + c;
            if (j >= n_feat) break;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                int64_t i = row0 + lane + 32 * u;
                double z = sB[c];
#pragma unroll
                for (int k = 0; k < FL_MAX_D; ++k)
                    if (k < d) z = fma(sW[c][k], xr[u][k], z);
                double sn, cs = 0.0;
                if (NEED_COS) sincos(z, &sn, &cs);
                else sn = sin(z);
                double val = sP[c] * sn;
                if (NEED_COS) val = fma(sQ[c], cs, val);
#pragma unroll
                for (int q = 0; q < NPP; ++q)
                    if (q < n_pp) val = fma(cpt[q][u] * sM[q][c], ((pp_cos_mask >> q) & 1) ? cs : sn, val);
                if (i < n_rows) A[j * ldA + row_offset + i] = val;
            }
        }
    }
}

// u_e = scale * sum_j beta_j sin(W_j.x_e + b_j), split over feature chunks;
// partial sums [split][n_eval] are reduced by k_eval_reduce in a fixed order.
constexpr int EVAL_SPLIT_COLS = 128;

__global__ void __launch_bounds__(128)
k_eval_partial(const double *__restrict__ x, int64_t n_eval, int d,
               const double *__restrict__ W, const double *__restrict__ b, int64_t n_feat,
               const double *__restrict__ beta, double *__restrict__ part)
{
    __shared__ double sW[EVAL_SPLIT_COLS][FL_MAX_D];
    __shared__ double sB[EVAL_SPLIT_COLS], sBeta[EVAL_SPLIT_COLS];
    const int64_t j0 = (int64_t)blockIdx.y * EVAL_SPLIT_COLS;
    const int ncols = (int)fl_min64(EVAL_SPLIT_COLS, n_feat - j0);
    for (int t = threadIdx.x; t < ncols; t += blockDim.x) {
        for (int k = 0; k < d; ++k) sW[t][k] = W[(j0 + t) * d + k];
        sB[t] = b[j0 + t];
        sBeta[t] = beta[j0 + t];
    }
    __syncthreads();
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_eval) return;
    double xe[FL_MAX_D];
    for (int k = 0; k < FL_MAX_D; ++k) xe[k] = (k < d) ? x[e * d + k] : 0.0;
    double acc = 0.0;
    for (int c = 0; c < ncols; ++c) {
        double z = sB[c];
        for (int k = 0; k < d; ++k) z = fma(sW[c][k], xe[k], z);
        acc = fma(sBeta[c], sin(z), acc);
    }
    part[(int64_t)blockIdx.y * n_eval + e] = acc;
}

__global__ void k_eval_reduce(const double *__restrict__ part, int nsplit, int64_t n_eval,
                              double scale, double *__restrict__ u)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_eval) return;
    double acc = 0.0;
    for (int s = 0; s < nsplit; ++s) acc += part[(int64_t)s * n_eval + e];
    u[e] = scale * acc;
}

// L[u](x_e) = sum_j beta_j (P_j sin z_ej + Q_j cos z_ej), z_ej = W_j.x_e + b_j, with the
// operator's column prefactors P, Q (eq. cyclic; scale included): split over feature
// chunks like k_eval_partial, the partial sums reduced by k_eval_reduce
__global__ void __launch_bounds__(128)
k_eval_op_partial(const double *__restrict__ x, int64_t n_eval, int d, const double *__restrict__ W,
                  const double *__restrict__ b, int64_t n_feat, const double *__restrict__ pref,
                  const double *__restrict__ beta, double *__restrict__ part)
{
    __shared__ double sW[EVAL_SPLIT_COLS][FL_MAX_D];
    __shared__ double sB[EVAL_SPLIT_COLS], sP[EVAL_SPLIT_COLS], sQ[EVAL_SPLIT_COLS];
    const int64_t j0 = (int64_t)blockIdx.y * EVAL_SPLIT_COLS;
    const int ncols = (int)fl_min64(EVAL_SPLIT_COLS, n_feat - j0);
    for (int t = threadIdx.x; t < ncols; t += blockDim.x) {
        for (int k = 0; k < d; ++k) sW[t][k] = W[(j0 + t) * d + k];
        sB[t] = b[j0 + t];
        sP[t] = beta[j0 + t] * pref[j0 + t];
        sQ[t] = beta[j0 + t] * pref[n_feat + j0 + t];
    }
    __syncthreads();
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_eval) return;
    double xe[FL_MAX_D];
    for (int k = 0; k < FL_MAX_D; ++k) xe[k] = (k < d) ? x[e * d + k] : 0.0;
    double acc = 0.0;
    for (int c = 0; c < ncols; ++c) {
        double z = sB[c];
        for (int k = 0; k < d; ++k) z = fma(sW[c][k], xe[k], z);
        double sn, cs;
        sincos(z, &sn, &cs);
        acc = fma(sP[c], sn, fma(sQ[c], cs, acc));
    }
    part[(int64_t)blockIdx.y * n_eval + e] = acc;
}

// grad_beta_j = scale * sum_e g_e sin(W_j.x_e + b_j): one feature per thread,
// points staged in shared memory in chunks (FP64).
constexpr int EA_PTS = 256;

__global__ void __launch_bounds__(128)
k_eval_adjoint(const double *__restrict__ x, int64_t n_eval, int d, const double *__restrict__ W,
               const double *__restrict__ b, int64_t n_feat, double scale,
               const double *__restrict__ g, double *__restrict__ grad)
{
    __shared__ double sx[EA_PTS][FL_MAX_D];
    __shared__ double sg[EA_PTS];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double w[FL_MAX_D];
    for (int k = 0; k < FL_MAX_D; ++k) w[k] = (j < n_feat && k < d) ? W[j * d + k] : 0.0;
    const double bj = (j < n_feat) ? b[j] : 0.0;
    double acc = 0.0;
    for (int64_t e0 = 0; e0 < n_eval; e0 += EA_PTS) {
        const int ne = (int)fl_min64(EA_PTS, n_eval - e0);
        __syncthreads();
        for (int t = threadIdx.x; t < ne; t += blockDim.x) {
            for (int k = 0; k < d; ++k) sx[t][k] = x[(e0 + t) * d + k];
            sg[t] = g[e0 + t];
        }
        __syncthreads();
        for (int e = 0; e < ne; ++e) {
            double z = bj;
            for (int k = 0; k < d; ++k) z = fma(w[k], sx[e][k], z);
            acc = fma(sg[e], sin(z), acc);
        }
    }
    if (j < n_feat) grad[j] = scale * acc;
}

// Manufactured sources and exact solutions (the problem catalogue of the
// header).  The sources are L[u*] worked out by hand for each u*.
struct fl_problem_params {
    double p[64];
    int n;
};

__global__ void k_rhs(int problem, int kind, fl_problem_params prm, const double *__restrict__ x,
                      int64_t n, int d, double weight, double *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *p = x + i * d;
    const double pi = 3.14159265358979323846;
    double v = 0.0;
    switch (problem) {
    case FASTLSQ_PROBLEM_POISSON_1D:
        if (kind == FASTLSQ_RHS_EXACT) v = sin(2 * pi * p[0]) + 0.5 * sin(6 * pi * p[0]);
        else v = 4 * pi * pi * sin(2 * pi * p[0]) + 18 * pi * pi * sin(6 * pi * p[0]);
        break;
    case FASTLSQ_PROBLEM_HELMHOLTZ_2D: {
        double s1 = sin(pi * p[0]) * sin(2 * pi * p[1]);
        double c1 = cos(3 * pi * p[0] + pi * p[1]);
        if (kind == FASTLSQ_RHS_EXACT) v = s1 + 0.3 * c1;
        else {
            double k2 = prm.p[0] * prm.p[0];
            v = (k2 - 5 * pi * pi) * s1 + 0.3 * (k2 - 10 * pi * pi) * c1;
        }
        break;
    }
    case FASTLSQ_PROBLEM_POISSON_5D: {
        double sum = 0.0, prod = 1.0;
        for (int k = 0; k < d; ++k) {
            sum += sin(pi * p[k]);
            prod *= p[k];
        }
        v = (kind == FASTLSQ_RHS_EXACT) ? sum + prod : pi * pi * sum;
        break;
    }
    case FASTLSQ_PROBLEM_NLPOISSON_2D:
    case FASTLSQ_PROBLEM_NLHELMHOLTZ_2D: {
        // u* = sin(pi x) sin(pi y) + x y / 2; Lap u* = -2 pi^2 sin(pi x) sin(pi y)
        const double sp = sin(pi * p[0]) * sin(pi * p[1]);
        const double us = sp + 0.5 * p[0] * p[1];
        if (kind == FASTLSQ_RHS_EXACT) v = us;
        else if (problem == FASTLSQ_PROBLEM_NLPOISSON_2D) v = 2 * pi * pi * sp + prm.p[0] * us * us * us;
        else v = -2 * pi * pi * sp + prm.p[0] * prm.p[0] * us + prm.p[1] * us * us * us;
        break;
    }
    case FASTLSQ_PROBLEM_VARCOEF_2D: {
        // div(nu grad u) = nu Lap u + grad nu . grad u with nu = 1 + a (x^2 + y^2/2) and
        // u* = sin(pi x) sin(2 pi y) + x y (Lap u* = -5 pi^2 sin(pi x) sin(2 pi y))
        const double a = prm.p[0];
        const double nu = 1.0 + a * (p[0] * p[0] + 0.5 * p[1] * p[1]);
        const double s2 = sin(pi * p[0]) * sin(2 * pi * p[1]);
        if (kind == FASTLSQ_RHS_EXACT) v = s2 + p[0] * p[1];
        else if (kind == FASTLSQ_RHS_COEF) v = nu;
        else if (kind == FASTLSQ_RHS_COEF_GRAD) v = 2.0 * a * p[0];
        else if (kind == FASTLSQ_RHS_COEF_GRAD + 1) v = a * p[1];
        else if (kind == FASTLSQ_RHS_SOURCE) {
            const double ux = pi * cos(pi * p[0]) * sin(2 * pi * p[1]) + p[1];
            const double uy = 2 * pi * sin(pi * p[0]) * cos(2 * pi * p[1]) + p[0];
            v = nu * (-5 * pi * pi * s2) + 2.0 * a * p[0] * ux + a * p[1] * uy;
        }
        break;
    }
    case FASTLSQ_PROBLEM_ALLEN_CAHN_1D:
        // tanh(k s) with k^2 = 1/(2 eps) solves eps u'' + u - u^3 = 0 (f = 0)
        if (kind == FASTLSQ_RHS_EXACT) v = tanh((p[0] - 0.5) / sqrt(2.0 * prm.p[0]));
        break;
    case FASTLSQ_PROBLEM_BURGERS_1D:
        // -tanh(k s) with k = 1/(2 nu) solves u u' - nu u'' = 0 (f = 0)
        if (kind == FASTLSQ_RHS_EXACT) v = -tanh((p[0] - 0.5) / (2.0 * prm.p[0]));
        break;
    case FASTLSQ_PROBLEM_GAUSS_SOURCE_2D:
        if (kind == FASTLSQ_RHS_SOURCE) {
            for (int k = 0; k + 3 < prm.n; k += 4) {
                double dx = p[0] - prm.p[k], dy = p[1] - prm.p[k + 1];
                v += prm.p[k + 3] * exp(-(dx * dx + dy * dy) / (2.0 * prm.p[k + 2] * prm.p[k + 2]));
            }
        }
        break;
    default:
        break;   // Bratu: f = 0, g = 0
    }
    out[i] = weight * v;
}

// dL/dtheta of the Gaussian source: per-thread partials over rows, fixed-order
// block reduction, then one partial per block [block][16] reduced on the host.
__global__ void __launch_bounds__(256)
k_source_grad(const double *__restrict__ x, int64_t n, fl_problem_params th, int n_src,
              const double *__restrict__ w, double *__restrict__ part)
{
    __shared__ double red[256];
    double acc[4 * 8];
    for (int q = 0; q < 4 * n_src; ++q) acc[q] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double px = x[2 * i], py = x[2 * i + 1];
        for (int k = 0; k < n_src; ++k) {
            const double *t = th.p + 4 * k;
            double dx = px - t[0], dy = py - t[1];
            double r2 = dx * dx + dy * dy, w2 = t[2] * t[2];
            double e = exp(-r2 / (2.0 * w2));
            acc[4 * k + 0] += w[i] * t[3] * e * dx / w2;
            acc[4 * k + 1] += w[i] * t[3] * e * dy / w2;
            acc[4 * k + 2] += w[i] * t[3] * e * r2 / (w2 * t[2]);
            acc[4 * k + 3] += w[i] * e;
        }
    }
    for (int q = 0; q < 4 * n_src; ++q) {
        red[threadIdx.x] = acc[q];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * 32 + q] = red[0];
        __syncthreads();
    }
}

bool op_needs_cos(const fl_op_params &op, unsigned *pp_cos_mask)
{
    bool need = false;
    for (int t = 0; t < op.n_terms; ++t) {
        int o = 0;
        for (int k = 0; k < op.d; ++k) o += op.alpha[t][k];
        if (o & 1) need = true;
    }
    unsigned mask = 0;
    for (int q = 0; q < op.n_pp; ++q) {
        int o = 0;
        for (int k = 0; k < op.d; ++k) o += op.pp_alpha[q][k];
        if (o & 1) {
            need = true;
            mask |= 1u << q;
        }
    }
    *pp_cos_mask = mask;
    return need;
}

}  // namespace

int fl_prefactors(fastlsq_ctx *ctx, const fl_op_params &op, const double *W, int64_t n_feat,
                  double scale, double row_weight, double *pref)
{
    FL_PROF(ctx, FASTLSQ_K_PREFACTOR);
    k_prefactors<<<(unsigned)fl_cdiv(n_feat, 128), 128, 0, ctx->stream>>>(op, W, n_feat,
                                                                          scale * row_weight, pref);
    FL_CHECK_LAUNCH(ctx, "prefactors");
    return 0;
}

int fl_launch_assemble_f32(fastlsq_ctx *ctx, const fl_op_params &op, const double *x,
                           int64_t n_rows, const double *W, const double *b, int64_t n_feat,
                           const double *pref, float *A, int64_t ldA, int64_t row_offset,
                           double)
{
    if (n_rows == 0 || n_feat == 0) return 0;
    unsigned mask;
    const bool need_cos = op_needs_cos(op, &mask);
    fl_pp_rows pp{};
    for (int q = 0; q < op.n_pp; ++q) pp.c[q] = op.pp_coef[q];
    const dim3 grid((unsigned)fl_cdiv(n_rows, AF_ROWS), (unsigned)fl_cdiv(n_feat, AF_COLS));
    const float c1 = ctx->cw2pi[0], c2 = ctx->cw2pi[1], c3 = ctx->cw2pi[2];
    FL_PROF(ctx, FASTLSQ_K_ASSEMBLE_F32);
#define FL_ASM32_PP(DD, COS, NPP)                                                                    \
    k_assemble_f32<DD, COS, NPP><<<grid, AF_THREADS, 0, ctx->stream>>>(                              \
        x, n_rows, W, b, n_feat, pref, op.n_pp, mask, pp, A, ldA, row_offset, c1, c2, c3)
#define FL_ASM32(DD)                                                                                 \
    case DD:                                                                                         \
        if (op.n_pp > 0) {                                                                           \
            if (need_cos) FL_ASM32_PP(DD, true, FL_MAX_PP);                                          \
            else FL_ASM32_PP(DD, false, FL_MAX_PP);                                                  \
        } else {                                                                                     \
            if (need_cos) FL_ASM32_PP(DD, true, 0);                                                  \
            else FL_ASM32_PP(DD, false, 0);                                                          \
        }                                                                                            \
        break;
    switch (op.d) {
        FL_ASM32(1) FL_ASM32(2) FL_ASM32(3) FL_ASM32(4) FL_ASM32(5) FL_ASM32(6) FL_ASM32(7) FL_ASM32(8)
    default: return fl_fail(ctx, FASTLSQ_ERR_INVALID, "assemble: dimension %d", op.d);
    }
#undef FL_ASM32
#undef FL_ASM32_PP
    FL_CHECK_LAUNCH(ctx, "assemble_f32");
    return 0;
}

int fl_launch_assemble_f64(fastlsq_ctx *ctx, const fl_op_params &op, const double *x,
                           int64_t n_rows, const double *W, const double *b, int64_t n_feat,
                           const double *pref, double *A, int64_t ldA, int64_t row_offset,
                           double)
{
    if (n_rows == 0 || n_feat == 0) return 0;
    unsigned mask;
    bool need_cos = op_needs_cos(op, &mask);
    fl_pp_rows pp{};
    for (int q = 0; q < op.n_pp; ++q) pp.c[q] = op.pp_coef[q];
    const int64_t ntiles = fl_cdiv(n_rows, ASM_ROWS) * fl_cdiv(n_feat, ASM_COLS);
    int64_t g = ntiles;
    if (ctx->asm64_ctas_per_sm > 0) g = std::min<int64_t>(g, (int64_t)ctx->num_sms * ctx->asm64_ctas_per_sm);
    if (g > INT32_MAX) g = INT32_MAX;
    const unsigned grid = (unsigned)g;
    FL_PROF(ctx, FASTLSQ_K_ASSEMBLE_F64);
#define FL_ASM64(COS, NPP)                                                                          \
    k_assemble_f64<COS, NPP><<<grid, ASM_THREADS, 0, ctx->stream>>>(                                \
        x, n_rows, op.d, W, b, n_feat, pref, op.n_pp, mask, pp, A, ldA, row_offset)
    // FP64: the four-slot form (per-point loop checked at run time) for every operator with
    // at most four per-point terms, plain operators included -- measured 684 us against 877 us
    // for a form without the loop on the helmholtz2d interior block -- and eight slots beyond
    if (op.n_pp > 4) {
        if (need_cos) FL_ASM64(true, FL_MAX_PP);
        else FL_ASM64(false, FL_MAX_PP);
    } else {
        if (need_cos) FL_ASM64(true, 4);
        else FL_ASM64(false, 4);
    }
#undef FL_ASM64
    FL_CHECK_LAUNCH(ctx, "assemble_f64");
    return 0;
}

int fl_launch_eval(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d, const double *W,
                   const double *b, int64_t n_feat, double scale, const double *beta, double *u)
{
    if (n_eval == 0) return 0;
    int nsplit = (int)fl_cdiv(n_feat, EVAL_SPLIT_COLS);
    double *part = (double *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(double) * nsplit * n_eval);
    if (!part) return FASTLSQ_ERR_NOMEM;
    dim3 grid((unsigned)fl_cdiv(n_eval, 128), (unsigned)nsplit);
    FL_PROF_N(ctx, FASTLSQ_K_EVAL, 2);
    k_eval_partial<<<grid, 128, 0, ctx->stream>>>(x, n_eval, d, W, b, n_feat, beta, part);
    FL_CHECK_LAUNCH(ctx, "eval_partial");
    k_eval_reduce<<<(unsigned)fl_cdiv(n_eval, 256), 256, 0, ctx->stream>>>(part, nsplit, n_eval,
                                                                           scale, u);
    FL_CHECK_LAUNCH(ctx, "eval_reduce");
    return 0;
}

int fl_launch_eval_op(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d, const double *W,
                      const double *b, int64_t n_feat, const double *pref, const double *beta, double *u)
{
    if (n_eval == 0) return 0;
    int nsplit = (int)fl_cdiv(n_feat, EVAL_SPLIT_COLS);
    double *part = (double *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(double) * nsplit * n_eval);
    if (!part) return FASTLSQ_ERR_NOMEM;
    dim3 grid((unsigned)fl_cdiv(n_eval, 128), (unsigned)nsplit);
    FL_PROF_N(ctx, FASTLSQ_K_EVAL, 2);
    k_eval_op_partial<<<grid, 128, 0, ctx->stream>>>(x, n_eval, d, W, b, n_feat, pref, beta, part);
    FL_CHECK_LAUNCH(ctx, "eval_op_partial");
    k_eval_reduce<<<(unsigned)fl_cdiv(n_eval, 256), 256, 0, ctx->stream>>>(part, nsplit, n_eval, 1.0, u);
    FL_CHECK_LAUNCH(ctx, "eval_reduce");
    return 0;
}

// ---------------------------------------------------------------------------
// fastlsq_eval_noalloc: the evaluation of fastlsq_eval with its partial sums in a
// fixed device array of this library instead of the context's workspace, so the
// call allocates nothing.  The array is shared by every context on a device; its
// address is looked up by fastlsq_create (fl_eval_static_lookup), with the context's
// device current, and kept in the context.
// ---------------------------------------------------------------------------
constexpr size_t FL_EVAL_STATIC_DOUBLES = (size_t)1 << 19;      // 4 MiB of FP64 partial sums
static __device__ __align__(256) double g_eval_static[FL_EVAL_STATIC_DOUBLES];

// The device address of the array in the current device's context.  Looking it up
// loads this library's device code (and commits the array) if that has not happened.
cudaError_t fl_eval_static_lookup(double **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_eval_static);
    *out = (e == cudaSuccess) ? (double *)p : nullptr;
    return e;
}

int fl_launch_eval_noalloc(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d, const double *W,
                           const double *b, int64_t n_feat, double scale, const double *beta, double *u)
{
    if (n_eval == 0) return 0;
    const int64_t nsplit = fl_cdiv(n_feat, EVAL_SPLIT_COLS);
    if (nsplit * n_eval > (int64_t)FL_EVAL_STATIC_DOUBLES)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID,
                       "eval_noalloc: ceil(n_feat/%d) * n_eval = %lld exceeds the %lld-entry static scratch",
                       EVAL_SPLIT_COLS, (long long)(nsplit * n_eval), (long long)FL_EVAL_STATIC_DOUBLES);
    double *part = ctx->eval_static;
    if (!part) return fl_fail(ctx, FASTLSQ_ERR_CUDA, "eval_noalloc: the scratch address was not found");
    dim3 grid((unsigned)fl_cdiv(n_eval, 128), (unsigned)nsplit);
    FL_PROF_N(ctx, FASTLSQ_K_EVAL, 2);
    k_eval_partial<<<grid, 128, 0, ctx->stream>>>(x, n_eval, d, W, b, n_feat, beta, part);
    FL_CHECK_LAUNCH(ctx, "eval_partial");
    k_eval_reduce<<<(unsigned)fl_cdiv(n_eval, 256), 256, 0, ctx->stream>>>(part, (int)nsplit, n_eval,
                                                                           scale, u);
    FL_CHECK_LAUNCH(ctx, "eval_reduce");
    return 0;
}

int fl_launch_eval_adjoint(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d,
                           const double *W, const double *b, int64_t n_feat, double scale,
                           const double *g, double *grad)
{
    FL_PROF(ctx, FASTLSQ_K_ADJOINT);
    k_eval_adjoint<<<(unsigned)fl_cdiv(n_feat, 128), 128, 0, ctx->stream>>>(x, n_eval, d, W, b, n_feat,
                                                                           scale, g, grad);
    FL_CHECK_LAUNCH(ctx, "eval_adjoint");
    return 0;
}

int fl_launch_rhs(fastlsq_ctx *ctx, int problem, int kind, const double *params, int n_params,
                  const double *x, int64_t n, int d, double weight, double *out)
{
    if (n == 0) return 0;
    fl_problem_params prm{};
    if (n_params > 64) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: at most 64 parameters");
    for (int i = 0; i < n_params; ++i) prm.p[i] = params[i];
    prm.n = n_params;
    FL_PROF(ctx, FASTLSQ_K_RHS);
    k_rhs<<<(unsigned)fl_cdiv(n, 256), 256, 0, ctx->stream>>>(problem, kind, prm, x, n, d, weight,
                                                              out);
    FL_CHECK_LAUNCH(ctx, "rhs");
    return 0;
}

int fl_launch_source_grad(fastlsq_ctx *ctx, const double *x, int64_t n, const double *theta,
                          int n_src, const double *w, double *dtheta_host)
{
    if (n_src < 1 || n_src > 8) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "source_grad: n_src 1..8");
    fl_problem_params th{};
    for (int i = 0; i < 4 * n_src; ++i) th.p[i] = theta[i];
    th.n = 4 * n_src;
    int nblk = (int)std::min<int64_t>(fl_cdiv(n, 256), 304);
    if (nblk < 1) nblk = 1;
    double *part = (double *)fl_ws(ctx, FL_WS_SCALARS, sizeof(double) * 32 * (nblk + 1));
    if (!part) return FASTLSQ_ERR_NOMEM;
    {
    FL_PROF(ctx, FASTLSQ_K_ADJOINT);
    k_source_grad<<<nblk, 256, 0, ctx->stream>>>(x, n, th, n_src, w, part);
    FL_CHECK_LAUNCH(ctx, "source_grad");
    }
    return fl_reduce_blocks_to_host(ctx, part, nblk, 32, 4 * n_src, dtheta_host);
}

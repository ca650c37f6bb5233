// Newton-Raphson for L[u] + N[u] = f with Dirichlet rows (Sec. 2.4, eq. newton).
//
// Once per call, in FP64: L64 (rows: interior L[phi_j](x_i); boundary
// bc_weight phi_j(x_i)) and H64 (interior phi_j(x_i)).  Every iteration:
//   residual   R = L64 beta + [N(H64 beta) - f; -bc_weight g]           (FP64)
//   Jacobian   J_ij = L[phi_j](x_i) + N'(u_i) phi_j(x_i), boundary rows
//              bc_weight phi_j: reassembled with the closed form on the GPU
//              (FP32 operator kernel with the per-point term N'(u_i) for the
//              MIXED factor; J64 = L64 + diag(N'(u)) H64 for refinement / FP64).
//              Burgers (N = lam u u_x0) adds a second per-point term on the
//              first-derivative feature: lam u_x0 phi_j + lam u d(phi_j)/dx_0, with
//              H1 = d(phi_j)/dx_0 at the interior points (FP64, once per call)
//   step       delta = argmin ||J delta + R||^2 + mu ||delta||^2
//   line search a = 1, 1/2, ... until ||R(beta + a delta)||^2 <= (1 - 2 c a) ||R||^2
//   stop       ||u(beta + a delta) - u(beta)|| / ||u(beta + a delta)|| <= tol
//              over the collocation rows (solution-level test).
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "qr.cuh"

int fl_matvec64(fastlsq_ctx *ctx, const double *A, int64_t ld, int64_t m, int64_t n,
                const double *v, double *out);

namespace {

__device__ __forceinline__ double nl_val(int kind, double lam, double u, double ux)
{
    if (kind == FASTLSQ_NL_EXP) return lam * exp(u);
    if (kind == FASTLSQ_NL_CUBIC) return lam * u * u * u;
    if (kind == FASTLSQ_NL_BURGERS) return lam * u * ux;
    return 0.0;
}

// R_i and u at the collocation rows from Lu = L64 beta (m), uh = H64 beta (n_int) and,
// for Burgers, uxh = H1 beta (n_int; null otherwise)
__global__ void k_newton_resid(const double *__restrict__ Lu, const double *__restrict__ uh,
                               const double *__restrict__ uxh, int64_t n_int, int64_t n_bc,
                               int kind, double lam, double bcw,
                               const double *__restrict__ f, const double *__restrict__ g,
                               double *__restrict__ R, double *__restrict__ u_rows)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_int) {
        R[i] = Lu[i] + nl_val(kind, lam, uh[i], uxh ? uxh[i] : 0.0) - f[i];
        u_rows[i] = uh[i];
    } else if (i < n_int + n_bc) {
        R[i] = Lu[i] - bcw * g[i - n_int];
        u_rows[i] = Lu[i] / bcw;
    }
}

// per-block partial sums of (R^2, (un - u)^2, un^2); fixed-order final sum
__global__ void __launch_bounds__(256)
k_newton_norms(const double *__restrict__ R, const double *__restrict__ un,
               const double *__restrict__ u, int64_t m, double *__restrict__ part)
{
    __shared__ double red[3][256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0, bq = 0, c = 0;
    if (i < m) {
        a = R[i] * R[i];
        double du = un[i] - u[i];
        bq = du * du;
        c = un[i] * un[i];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = bq;
    red[2][threadIdx.x] = c;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = red[q][0];
}

__global__ void k_sum3(const double *__restrict__ part, int nblk, double *__restrict__ out)
{
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[3 * b + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// derivative of N in the direction phi: c0 phi + c1 d(phi)/dx_0 (c1 only for Burgers)
__global__ void k_nl_prime(const double *__restrict__ uh, const double *__restrict__ uxh, int64_t n,
                           int kind, double lam, double *__restrict__ c0, double *__restrict__ c1)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double u = uh[i];
    double a = 0.0;
    if (kind == FASTLSQ_NL_EXP) a = lam * exp(u);
    else if (kind == FASTLSQ_NL_CUBIC) a = 3.0 * lam * u * u;
    else if (kind == FASTLSQ_NL_BURGERS) {
        a = lam * uxh[i];
        c1[i] = lam * u;
    }
    c0[i] = a;
}

// J64 = L64 + diag(c0) H64 (+ diag(c1) H1) on the interior rows (boundary rows copied)
__global__ void k_jacobian64(const double *__restrict__ L64, const double *__restrict__ H64,
                             const double *__restrict__ c0, const double *__restrict__ H1,
                             const double *__restrict__ c1, int64_t n_int, int64_t m, int64_t n,
                             int64_t ld, double *__restrict__ J)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y;
    if (i >= m || j >= n) return;
    double v = L64[i + j * ld];
    if (i < n_int) {
        v = fma(c0[i], H64[i + j * n_int], v);
        if (H1) v = fma(c1[i], H1[i + j * n_int], v);
    }
    J[i + j * ld] = v;
}

__global__ void k_axpy_neg(const double *__restrict__ beta, const double *__restrict__ delta,
                           double a, int64_t n, double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = beta[i] + a * delta[i];
}

__global__ void k_neg(const double *__restrict__ x, int64_t n, double *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = -x[i];
}

struct NewtonBufs {
    double *L64, *H64, *H1, *J64;   // H1: Burgers only
    float *J32;
    double *Lu, *uh, *uxh, *R, *Rn, *u, *un, *c, *c1, *delta, *bt, *negR, *part, *sums;
};

}  // namespace

static int newton_residual(fastlsq_ctx *ctx, const fastlsq_newton_problem *p, int64_t n,
                           const NewtonBufs &B, const double *beta, double *R, double *u_rows)
{
    const int64_t m = p->n_int + p->n_bc;
    FL_TRY(fl_matvec64(ctx, B.L64, m, m, n, beta, B.Lu));
    FL_TRY(fl_matvec64(ctx, B.H64, p->n_int, p->n_int, n, beta, B.uh));
    if (B.H1) FL_TRY(fl_matvec64(ctx, B.H1, p->n_int, p->n_int, n, beta, B.uxh));
    FL_PROF(ctx, FASTLSQ_K_NEWTON);
    k_newton_resid<<<(unsigned)fl_cdiv(m, 256), 256, 0, ctx->stream>>>(
        B.Lu, B.uh, B.H1 ? B.uxh : nullptr, p->n_int, p->n_bc, p->nl_kind, p->nl_lam,
        p->bc_weight, p->f, p->g, R, u_rows);
    FL_CHECK_LAUNCH(ctx, "newton_resid");
    return 0;
}

// host copy of (||R||^2, ||un - u||^2, ||un||^2)
static int newton_norms(fastlsq_ctx *ctx, int64_t m, const NewtonBufs &B, const double *R,
                        const double *un, const double *u, double out[3])
{
    int nblk = (int)fl_cdiv(m, 256);
    FL_PROF_N(ctx, FASTLSQ_K_NEWTON, 2);
    k_newton_norms<<<nblk, 256, 0, ctx->stream>>>(R, un, u, m, B.part);
    FL_CHECK_LAUNCH(ctx, "newton_norms");
    k_sum3<<<1, 32, 0, ctx->stream>>>(B.part, nblk, B.sums);
    FL_CHECK_LAUNCH(ctx, "newton_sum3");
    cudaError_t e = cudaMemcpyAsync(out, B.sums, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "newton readback");
    return 0;
}

extern "C" int fastlsq_newton(fastlsq_ctx *ctx, const fastlsq_newton_problem *p, const double *W,
                              const double *b, int64_t n_feat, double scale,
                              const fastlsq_newton_opts *o, double *beta_io,
                              fastlsq_newton_stats *stats)
{
    if (!ctx || !p || !o || !W || !b || !beta_io) return FASTLSQ_ERR_INVALID;
    if (p->n_int < 1 || p->n_bc < 0 || !p->x_int || !p->f || (p->n_bc > 0 && (!p->x_bc || !p->g)))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton: bad problem");
    if (p->op.n_pp != 0) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton: operator has per-point terms");
    if (o->max_iter < 1 || o->max_iter > 64 || o->max_halvings < 0 || o->max_halvings > 60 ||
        !(p->bc_weight > 0) || o->mu < 0)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton: bad options");
    if (o->prec != FASTLSQ_PREC_FP64 && o->prec != FASTLSQ_PREC_MIXED)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton: precision");
    if (p->nl_kind < FASTLSQ_NL_NONE || p->nl_kind > FASTLSQ_NL_BURGERS)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton: unknown nonlinearity %d", (int)p->nl_kind);
    const bool burgers = (p->nl_kind == FASTLSQ_NL_BURGERS);
    fl_op_params opL;
    FL_TRY(fl_pack_op(ctx, &p->op, &opL));
    if (opL.d != p->d) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton: op.d != d");
    const int64_t n = n_feat, n_int = p->n_int, n_bc = p->n_bc, m = n_int + n_bc;
    const int d = p->d;

    // identity operator (alpha = 0) for the basis rows
    fl_op_params opI;
    memset(&opI, 0, sizeof(opI));
    opI.d = d;
    opI.n_terms = 1;
    opI.coef[0] = 1.0;
    // first derivative along x_0 (Burgers' advection feature)
    fl_op_params opD = opI;
    opD.alpha[0][0] = 1;

    // buffers
    NewtonBufs B{};
    int rc = 0;
    auto alloc = [&](size_t bytes) -> void * {
        void *ptr = nullptr;
        if (rc) return nullptr;
        cudaError_t e = cudaMallocAsync(&ptr, bytes ? bytes : 16, ctx->stream);
        if (e != cudaSuccess) {
            rc = fl_cuda(ctx, e, "newton allocation");
            return nullptr;
        }
        return ptr;
    };
    B.L64 = (double *)alloc(sizeof(double) * m * n);
    B.H64 = (double *)alloc(sizeof(double) * n_int * n);
    B.H1 = burgers ? (double *)alloc(sizeof(double) * n_int * n) : nullptr;
    B.uxh = burgers ? (double *)alloc(sizeof(double) * n_int) : nullptr;
    B.c1 = burgers ? (double *)alloc(sizeof(double) * n_int) : nullptr;
    B.J64 = (double *)alloc(sizeof(double) * m * n);
    B.J32 = (o->prec == FASTLSQ_PREC_MIXED) ? (float *)alloc(sizeof(float) * m * n) : nullptr;
    B.Lu = (double *)alloc(sizeof(double) * m);
    B.uh = (double *)alloc(sizeof(double) * n_int);
    B.R = (double *)alloc(sizeof(double) * m);
    B.Rn = (double *)alloc(sizeof(double) * m);
    B.u = (double *)alloc(sizeof(double) * m);
    B.un = (double *)alloc(sizeof(double) * m);
    B.c = (double *)alloc(sizeof(double) * n_int);
    B.delta = (double *)alloc(sizeof(double) * n);
    B.bt = (double *)alloc(sizeof(double) * n);
    B.negR = (double *)alloc(sizeof(double) * m);
    B.part = (double *)alloc(sizeof(double) * 3 * (fl_cdiv(m, 256) + 1));
    B.sums = (double *)alloc(sizeof(double) * 4);
    double *beta = (double *)alloc(sizeof(double) * n);
    double *pref = (double *)alloc(sizeof(double) * (2 + FL_MAX_PP) * n);
    fastlsq_newton_stats st;
    memset(&st, 0, sizeof(st));
    int status = FASTLSQ_WARN_MAXITER;
    int it = 0;
    double h3[3];
    double rr = 0.0;
    if (rc) goto cleanup;

    // FP64 operator rows, once
#define NT_TRY(expr)                      \
    do {                                  \
        int _r = (expr);                  \
        if (_r < 0) { rc = _r; goto cleanup; } \
    } while (0)
    NT_TRY(fl_prefactors(ctx, opL, W, n, scale, 1.0, pref));
    NT_TRY(fl_launch_assemble_f64(ctx, opL, p->x_int, n_int, W, b, n, pref, B.L64, m, 0, 1.0));
    NT_TRY(fl_prefactors(ctx, opI, W, n, scale, p->bc_weight, pref));
    NT_TRY(fl_launch_assemble_f64(ctx, opI, p->x_bc, n_bc, W, b, n, pref, B.L64, m, n_int, p->bc_weight));
    NT_TRY(fl_prefactors(ctx, opI, W, n, scale, 1.0, pref));
    NT_TRY(fl_launch_assemble_f64(ctx, opI, p->x_int, n_int, W, b, n, pref, B.H64, n_int, 0, 1.0));
    if (burgers) {
        NT_TRY(fl_prefactors(ctx, opD, W, n, scale, 1.0, pref));
        NT_TRY(fl_launch_assemble_f64(ctx, opD, p->x_int, n_int, W, b, n, pref, B.H1, n_int, 0, 1.0));
    }
    if (cudaMemcpyAsync(beta, beta_io, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream) !=
        cudaSuccess) {
        rc = fl_cuda(ctx, cudaGetLastError(), "newton copy");
        goto cleanup;
    }

    NT_TRY(newton_residual(ctx, p, n, B, beta, B.R, B.u));
    NT_TRY(newton_norms(ctx, m, B, B.R, B.u, B.u, h3));
    rr = h3[0];
    for (it = 0; it < o->max_iter; ++it) {
        st.res_norm[it] = sqrt(rr);
        // Jacobian with the per-point coefficient N'(u_i)
        {
        FL_PROF_N(ctx, FASTLSQ_K_NEWTON, 3);
        k_nl_prime<<<(unsigned)fl_cdiv(n_int, 256), 256, 0, ctx->stream>>>(
            B.u, B.uxh, n_int, p->nl_kind, p->nl_lam, B.c, B.c1);
        k_jacobian64<<<dim3((unsigned)fl_cdiv(m, 256), (unsigned)n), 256, 0, ctx->stream>>>(
            B.L64, B.H64, B.c, B.H1, B.c1, n_int, m, n, m, B.J64);
        k_neg<<<(unsigned)fl_cdiv(m, 256), 256, 0, ctx->stream>>>(B.R, m, B.negR);
        }
        if (cudaGetLastError() != cudaSuccess) {
            rc = fl_fail(ctx, FASTLSQ_ERR_CUDA, "newton kernels");
            goto cleanup;
        }
        if (o->prec == FASTLSQ_PREC_MIXED) {
            fl_op_params opJ = opL;
            opJ.n_pp = 1;
            memset(opJ.pp_alpha, 0, sizeof(opJ.pp_alpha));
            opJ.pp_coef[0] = B.c;    // alpha = 0 per-point term N'(u_i) phi_j
            if (burgers) {           // lam u_i d(phi_j)/dx_0
                opJ.n_pp = 2;
                opJ.pp_alpha[1][0] = 1;
                opJ.pp_coef[1] = B.c1;
            }
            NT_TRY(fl_prefactors(ctx, opJ, W, n, scale, 1.0, pref));
            NT_TRY(fl_launch_assemble_f32(ctx, opJ, p->x_int, n_int, W, b, n, pref, B.J32, m, 0, 1.0));
            NT_TRY(fl_prefactors(ctx, opI, W, n, scale, p->bc_weight, pref));
            NT_TRY(fl_launch_assemble_f32(ctx, opI, p->x_bc, n_bc, W, b, n, pref, B.J32, m, n_int,
                                          p->bc_weight));
            NT_TRY(fastlsq_lstsq(ctx, FASTLSQ_PREC_MIXED, B.J32, FASTLSQ_F32, m, m, n, o->mu, B.negR,
                                 1, m, B.delta, n, B.J64, m, o->max_refine, FASTLSQ_REFINE_CGLS,
                                 o->refine_tol > 0 ? o->refine_tol : 1e-10, nullptr, nullptr));
        } else {
            NT_TRY(fastlsq_lstsq(ctx, FASTLSQ_PREC_FP64, B.J64, FASTLSQ_F64, m, m, n, o->mu, B.negR,
                                 1, m, B.delta, n, nullptr, 0, 0, FASTLSQ_REFINE_CLASSICAL, 0.0,
                                 nullptr, nullptr));
        }
        // backtracking line search on ||R||
        double a = 1.0, rr_new = 0.0;
        bool accepted = false;
        for (int h = 0; h <= o->max_halvings; ++h) {
            ctx->prof.launches[FASTLSQ_K_NEWTON] += 1;
            k_axpy_neg<<<(unsigned)fl_cdiv(n, 256), 256, 0, ctx->stream>>>(beta, B.delta, a, n, B.bt);
            NT_TRY(newton_residual(ctx, p, n, B, B.bt, B.Rn, B.un));
            NT_TRY(newton_norms(ctx, m, B, B.Rn, B.un, B.u, h3));
            rr_new = h3[0];
            if (std::isfinite(rr_new) && rr_new <= (1.0 - 2.0 * o->armijo_c * a) * rr) {
                accepted = true;
                break;
            }
            a *= 0.5;
        }
        if (!accepted) {
            status = FASTLSQ_WARN_LINESEARCH;
            break;
        }
        st.alpha[it] = a;
        st.step_rel[it] = (h3[2] > 0) ? sqrt(h3[1] / h3[2]) : INFINITY;
        std::swap(beta, B.bt);
        std::swap(B.R, B.Rn);
        std::swap(B.u, B.un);
        rr = rr_new;
        if (sqrt(h3[1]) <= o->tol * sqrt(h3[2])) {
            status = 0;
            ++it;
            break;
        }
    }
    st.res_norm[it] = sqrt(rr);
    st.iters = it;
    st.status = status;
    if (cudaMemcpyAsync(beta_io, beta, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream) !=
        cudaSuccess)
        rc = fl_fail(ctx, FASTLSQ_ERR_CUDA, "newton result copy");
    if (stats) *stats = st;
#undef NT_TRY
cleanup:
    {
        void *ptrs[] = {B.L64, B.H64, B.H1, B.J64, B.J32, B.Lu, B.uh, B.uxh, B.R, B.Rn, B.u, B.un,
                        B.c, B.c1, B.delta, B.bt, B.negR, B.part, B.sums, beta, pref};
        for (void *q : ptrs)
            if (q) cudaFreeAsync(q, ctx->stream);
    }
    if (rc < 0) return rc;
    int frc = fastlsq_sync(ctx);
    if (frc < 0) return frc;
    return status;
}

// Continuation (homotopy) of Sec. 2.4: a sequence of Newton solves whose interior
// operator coefficients move stage by stage towards the target problem (e.g. the
// viscosity of steady Burgers 1.0 -> 0.5 -> 0.2 -> 0.1), each warm-started from the
// previous stage's solution.
extern "C" int fastlsq_newton_continuation(fastlsq_ctx *ctx, const fastlsq_newton_problem *p,
                                           const double *W, const double *b, int64_t n_feat,
                                           double scale, const fastlsq_newton_opts *o,
                                           int32_t n_stages, const double *stage_coef,
                                           double *beta_io, fastlsq_newton_stats *stats)
{
    if (!ctx || !p) return FASTLSQ_ERR_INVALID;
    if (n_stages < 1 || n_stages > 64 || !stage_coef)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton_continuation: 1..64 stages with coefficients");
    const int nt = p->op.n_terms;
    if (nt < 1 || nt > FL_MAX_TERMS)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "newton_continuation: operator terms");
    std::vector<double> coef((size_t)nt);
    fastlsq_newton_problem q = *p;
    q.op.coef = coef.data();
    int status = 0;
    for (int k = 0; k < n_stages; ++k) {
        for (int t = 0; t < nt; ++t) coef[t] = stage_coef[(size_t)k * nt + t];
        status = fastlsq_newton(ctx, &q, W, b, n_feat, scale, o, beta_io, stats ? &stats[k] : nullptr);
        if (status < 0 || status == FASTLSQ_WARN_LINESEARCH) break;
    }
    return status;
}

/*
 * fastlsq.h -- C ABI of the GB300 (sm_103a) FastLSQ hot path.
 *
 * The method (arXiv 2602.10541): u(x) = s * sum_j beta_j sin(W_j.x + b_j) with
 * s = 1/sqrt(N) (Sec. 2.1, eq. approximation); every linear operator applied to
 * a feature has the closed form D^alpha phi_j = (prod_k W_jk^alpha_k) *
 * Phi_{|alpha| mod 4}(W_j.x + b_j), Phi = (sin, cos, -sin, -cos) (Sec. 2.2,
 * eq. cyclic); a linear PDE becomes the least-squares problem
 * [A_pde; lambda A_bc] beta = [f; lambda g] (Sec. 2.3, eq. linear_system,
 * Alg. 1); a nonlinear one is solved by Newton-Raphson with Tikhonov-regularised
 * least-squares steps (Sec. 2.4, eq. newton); gradients flow through the
 * pre-factored solve (Sec. 2.5, Sec. 3.8).
 *
 * Conventions for every entry point:
 *  - All array arguments are DEVICE pointers on the context's device unless the
 *    argument says "host".  The caller owns every array; the library owns only
 *    the context and factor handles, released by their _destroy calls.
 *  - Matrices are column-major with a leading dimension ld >= rows; vectors are
 *    contiguous.  Points x are row-major [n][d]; feature weights W are row-major
 *    [n_feat][d]; biases b are [n_feat].  x, W, b, right-hand sides and
 *    coefficients are double precision; the operator matrix may be float or
 *    double (fastlsq_dtype).
 *  - Work is queued on the context's stream and is asynchronous unless the call
 *    documents a host read-back (the stats structs).  Call with the context's
 *    device current on the calling thread (fastlsq_create leaves it current).
 *  - Return value: 0 success; negative = error (-1 invalid argument, -2 out of
 *    memory, -3 CUDA error, -4 device-side wait timed out, -5 non-finite value);
 *    positive = warning (1 Newton reached max_iter, 2 line search failed,
 *    3 numerically rank-deficient R).  No exception or abort crosses the ABI;
 *    fastlsq_last_error() gives a message.
 *  - Sizes: n_feat <= 16384, d <= 8, at most 32 operator terms, per-point terms
 *    <= 4; n_rows is limited by device memory and by the panel kernel's on-chip
 *    capacity (fastlsq_lstsq returns -1 with a message when exceeded).
 */
#ifndef FASTLSQ_H
#define FASTLSQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FASTLSQ_API __attribute__((visibility("default")))
#else
#define FASTLSQ_API
#endif

#define FASTLSQ_OK 0
#define FASTLSQ_ERR_INVALID (-1)
#define FASTLSQ_ERR_NOMEM (-2)
#define FASTLSQ_ERR_CUDA (-3)
#define FASTLSQ_ERR_TIMEOUT (-4)
#define FASTLSQ_ERR_NONFINITE (-5)
#define FASTLSQ_WARN_MAXITER 1
#define FASTLSQ_WARN_LINESEARCH 2
#define FASTLSQ_WARN_RANKDEF 3

typedef struct fastlsq_ctx fastlsq_ctx;        /* device, stream, workspace, tile table */
typedef struct fastlsq_factor fastlsq_factor;  /* checkpointed QR factors (reusable)    */

typedef enum { FASTLSQ_F32 = 0, FASTLSQ_F64 = 1 } fastlsq_dtype;

/* Solve precision.  FP64: FP64 operator, FP64 Householder QR (panel and trailing
 * updates), FP64 triangular solve.  MIXED: FP32 operator, FP32 panels, trailing
 * updates as split TF32x3 tensor-core products with FP32 accumulation (SIMT FP32
 * when tensor-core updates are disabled), then classical iterative refinement:
 * FP64 residual r = rhs - A64 beta against a caller-supplied FP64 operator, the
 * correction R^{-1} Q^T r solved with the FP32 factors, beta accumulated in
 * FP64. */
typedef enum { FASTLSQ_PREC_FP64 = 0, FASTLSQ_PREC_MIXED = 1 } fastlsq_prec;

/* Refinement of a MIXED solve.  CLASSICAL: beta += R^{-1} Q^T (rhs - A64 beta),
 * max_refine times (0..7); converges when the least-squares residual is small
 * (consistent systems such as the manufactured linear PDEs).  CGLS: CGLS on the
 * FP64 operator right-preconditioned by the factor's R, started from the direct
 * solve, at most max_refine iterations (0..64) or until the preconditioned
 * normal-equation residual falls by refine_tol; converges also for
 * large-residual and ill-conditioned systems (Newton steps, inverse problems). */
typedef enum { FASTLSQ_REFINE_CLASSICAL = 0, FASTLSQ_REFINE_CGLS = 1 } fastlsq_refine;

/* A linear operator as a list of terms sum_t coef[t] D^{alpha_t} (the paper's Op,
 * App. B).  alpha: host [n_terms][d] multi-indices; coef: host [n_terms].
 * pp_*: optional per-point terms (at most 8) whose coefficient varies by row:
 * term q adds pp_coef[q][i] * D^{pp_alpha_q} phi_j(x_i), pp_coef[q] a DEVICE
 * double array of n_rows entries (the rows of this call).  This is how the
 * Newton Jacobian's N'(u_i) phi_j enters (eq. newton), and how a variable-
 * coefficient operator such as div(nu grad u) = nu Lap u + grad nu . grad u
 * (Sec. 3.8, coil localisation) is written: 2d per-point terms with coefficients
 * nu(x_i) on D^{2e_k} and d nu/dx_k(x_i) on D^{e_k}. */
typedef struct {
    int32_t d;
    int32_t n_terms;
    const int32_t *alpha;          /* host [n_terms * d] */
    const double *coef;            /* host [n_terms]     */
    int32_t n_pp;                  /* number of per-point terms (0..8) */
    const int32_t *pp_alpha;       /* host [n_pp * d]    */
    const double *const *pp_coef;  /* host array of n_pp DEVICE pointers */
} fastlsq_op;

/* Create a context on `device` that queues work on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  Returns 0 or an error. */
FASTLSQ_API int fastlsq_create(fastlsq_ctx **ctx, int device, void *cuda_stream);
/* Release the context and its workspace (waits for its stream first). */
FASTLSQ_API int fastlsq_destroy(fastlsq_ctx *ctx);
/* Replace the stream the context queues work on. */
FASTLSQ_API int fastlsq_set_stream(fastlsq_ctx *ctx, void *cuda_stream);
/* Make every later call on this context that reads a factor's FP64 operator
 * A_refine (the refinement residuals of fastlsq_lstsq / fastlsq_factor_solve, the
 * PCG products and A v of fastlsq_backward) first make the context's stream wait
 * for `cuda_event` (a cudaEvent_t), as cudaStreamWaitEvent does at that point:
 * the wait binds to the event's latest record made before the call.  The FP64
 * operator can then be assembled on another stream while the FP32 factorisation
 * runs; only the refinement waits for it.  NULL removes the wait.  The event is
 * not owned by the context and must outlive its use. */
FASTLSQ_API int fastlsq_set_refine_event(fastlsq_ctx *ctx, void *cuda_event);
/* Message describing the last error on this context ("" if none). Owned by ctx. */
FASTLSQ_API const char *fastlsq_last_error(const fastlsq_ctx *ctx);
/* Synchronise the context's stream and return the first device-side error flag
 * raised since the last call (0 if none), then clear it. */
FASTLSQ_API int fastlsq_sync(fastlsq_ctx *ctx);

/*
 * Assemble one row block of the operator matrix (Sec. 2.3 eq. linear_system,
 * Alg. 1 steps 3-4) with the cyclic-derivative closed form (eq. cyclic):
 *
 *   A[(row_offset + i) + j*ldA] = row_weight * scale *
 *        sum_t (coef_t + pp) * (prod_k W_jk^alpha_tk) * Phi_{|alpha_t| mod 4}(W_j.x_i + b_j)
 *
 * for i < n_rows, j < n_feat.  x: [n_rows][op->d] (double), W: [n_feat][d]
 * (double), b: [n_feat] (double).  A: dtype F32 or F64, column-major, ldA >=
 * row_offset + n_rows; rows outside [row_offset, row_offset + n_rows) are not
 * touched.  The F32 path rounds x, W, b to float, reduces the argument with a
 * three-part 2 pi (Cody-Waite) and evaluates sin/cos on the SFU; the F64 path
 * uses double-precision sin/cos.  Interior rows use the PDE operator with
 * row_weight 1; boundary rows the boundary operator with row_weight = lambda.
 */
FASTLSQ_API int fastlsq_assemble(fastlsq_ctx *ctx, fastlsq_dtype dtype,
                     const double *x, int64_t n_rows, const fastlsq_op *op,
                     double row_weight, const double *W, const double *b,
                     int64_t n_feat, double scale,
                     void *A, int64_t ldA, int64_t row_offset);

/* Problem ids for fastlsq_rhs (the manufactured and synthetic problems). */
typedef enum {
    FASTLSQ_PROBLEM_POISSON_1D = 1,    /* -u'' = f, u* = sin(2 pi x) + 0.5 sin(6 pi x)              */
    FASTLSQ_PROBLEM_HELMHOLTZ_2D = 2,  /* Lap u + k^2 u = f, params[0] = k,                         */
                                       /* u* = sin(pi x) sin(2 pi y) + 0.3 cos(3 pi x + pi y)       */
    FASTLSQ_PROBLEM_POISSON_5D = 3,    /* -Lap u = f, u* = sum_k sin(pi x_k) + prod_k x_k           */
    FASTLSQ_PROBLEM_BRATU_2D = 4,      /* Lap u + lam e^u = 0, u = 0 on the boundary (f = g = 0)    */
    FASTLSQ_PROBLEM_NLPOISSON_2D = 6,  /* -Lap u + lam u^3 = f, params[0] = lam (Sec. 3.3 NL-Poisson;  */
                                       /* u* = sin(pi x) sin(pi y) + x y / 2, Dirichlet data u*)      */
    FASTLSQ_PROBLEM_NLHELMHOLTZ_2D = 7, /* Lap u + k^2 u + lam u^3 = f, params = (k, lam) (Sec. 3.3  */
                                       /* NL-Helmholtz; the same u*)                                  */
    FASTLSQ_PROBLEM_ALLEN_CAHN_1D = 8, /* eps u'' + u - u^3 = 0 on [0,1], params[0] = eps (Sec. 3.3   */
                                       /* Allen-Cahn; f = 0), u* = tanh((x - 1/2) / sqrt(2 eps))     */
    FASTLSQ_PROBLEM_BURGERS_1D = 9,    /* u u' - nu u'' = 0 on [0,1], params[0] = nu (Sec. 3.3 steady */
                                       /* Burgers; f = 0), u* = -tanh((x - 1/2) / (2 nu))            */
    FASTLSQ_PROBLEM_VARCOEF_2D = 10,   /* div(nu grad u) = f on [0,1]^2 (Sec. 3.8's variable-          */
                                       /* coefficient form), nu = 1 + a (x^2 + y^2/2), params[0] = a, */
                                       /* u* = sin(pi x) sin(2 pi y) + x y; kinds COEF / COEF_GRAD    */
                                       /* give nu and its gradient at points                           */
    FASTLSQ_PROBLEM_GAUSS_SOURCE_2D = 5 /* -Lap u = sum_k a_k exp(-|x-c_k|^2/(2 w_k^2)), params =   */
                                       /* theta [n_src][4] = (c_x, c_y, w, a)                      */
} fastlsq_problem;

/* SOURCE: f; EXACT: u*; COEF: the variable coefficient nu of the problem's operator;
 * COEF_GRAD + k: d nu / d x_k (problems with a variable coefficient only). */
typedef enum { FASTLSQ_RHS_SOURCE = 0, FASTLSQ_RHS_EXACT = 1, FASTLSQ_RHS_COEF = 2,
               FASTLSQ_RHS_COEF_GRAD = 3 } fastlsq_rhs_kind;

/*
 * Right-hand side entries (eq. linear_system): out[i] = weight * f(x_i)
 * (kind SOURCE, the interior equation's source) or weight * u*(x_i) (kind EXACT,
 * the Dirichlet data g and the reference solution for error measurement; 0 for
 * problems without a closed form).  params: host [n_params].  x: [n][d].
 */
FASTLSQ_API int fastlsq_rhs(fastlsq_ctx *ctx, fastlsq_problem problem, fastlsq_rhs_kind kind,
                const double *params, int32_t n_params, const double *x, int64_t n,
                int32_t d, double weight, double *out);

/*
 * Evaluate a linear operator of the approximation at points (eq. cyclic applied to
 * u = scale * sum_j beta_j sin(W_j.x + b_j)): u[e] = (L u)(x_e) for the operator L of
 * `op` (terms c_t D^{alpha_t}), e.g. a gradient component (one term, alpha = e_k), the
 * Laplacian, or the PDE residual's linear part; FP64.  Per-point coefficients
 * (op->n_pp > 0) are not allowed (they belong to collocation rows).  x: [n_eval][d]
 * with d = op->d; W: [n_feat][d]; b, beta: [n_feat]; u: [n_eval] (all device).
 * Errors: FASTLSQ_ERR_INVALID for bad sizes, null arrays or per-point terms.
 */
FASTLSQ_API int fastlsq_eval_op(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                                const fastlsq_op *op, const double *W, const double *b, int64_t n_feat,
                                double scale, const double *beta, double *u);

/*
 * Evaluate the approximation at points (eq. approximation, Alg. 1 return line):
 * u[e] = scale * sum_j beta[j] sin(W_j.x_e + b_j) for e < n_eval, in FP64.
 * x: [n_eval][d].  Used for test-set errors and sensor readouts.
 */
FASTLSQ_API int fastlsq_eval(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                 const double *W, const double *b, int64_t n_feat, double scale,
                 const double *beta, double *u);

/*
 * fastlsq_eval without any device allocation.  The paper has no counterpart: this
 * entry serves callers that cannot call cudaMalloc while they run, for example a
 * service that reserves all of its device memory at start-up and must not fail or
 * stall on an allocation in the middle of a request, or code running inside a
 * custom device allocator's own callbacks, where allocating again would re-enter
 * the allocator.  fastlsq_eval may grow the context's workspace with cudaMalloc;
 * this call never does.
 *
 * Arguments, layout and result are those of fastlsq_eval, and the result is
 * bitwise the same (the same kernels in the same order).  The only difference is
 * where the scratch lives: the FP64 partial sums, ceil(n_feat / 128) x n_eval of
 * them, are written into a fixed 4 MiB array compiled into this library (524,288
 * doubles) instead of the context's workspace.  So the call requires
 * ceil(n_feat / 128) * n_eval <= 524288 (for example 5000 points with up to 13,312
 * features) and returns FASTLSQ_ERR_INVALID, without launching anything, when the
 * request is larger.  Nothing in the array needs to start at zero: every entry a
 * call reads was written earlier in the same call.
 *
 * The array's device address is looked up with cudaGetSymbolAddress when the context
 * is created (fastlsq_create, with the context's device current); that lookup also
 * loads the library's device code, so the array is committed at context creation, not
 * at the first call: create the context before reserving the rest of the device's
 * memory.  A context does not outlive a device reset (create a new one after
 * cudaDeviceReset; it looks the array up again).  n_feat above 16384 returns
 * FASTLSQ_ERR_INVALID like fastlsq_eval.  There is one array per device for the whole process: two calls whose
 * executions can overlap (different streams, host threads or contexts on the same
 * device) use the same scratch and give wrong results.  Serialise them.
 */
FASTLSQ_API int fastlsq_eval_noalloc(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                         const double *W, const double *b, int64_t n_feat, double scale,
                         const double *beta, double *u);

/*
 * Adjoint of fastlsq_eval (the sensor readout u_s = H_s beta of Sec. 3.8):
 * grad_beta[j] = scale * sum_e g[e] sin(W_j.x_e + b_j), FP64.  x: [n_eval][d],
 * g: [n_eval], grad_beta: [n_feat].
 */
FASTLSQ_API int fastlsq_eval_adjoint(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                                     const double *W, const double *b, int64_t n_feat, double scale,
                                     const double *g, double *grad_beta);

typedef struct {
    int32_t refine_steps;      /* refinement steps / CGLS iterations performed     */
    int32_t nb;                /* panel width used                                 */
    int32_t tensor_core;       /* trailing-update mode of the factor: 0 SIMT, 1 outer
                                  blocks on tcgen05 (bf16 three-part split), 2 panel
                                  by panel on tcgen05 (TF32x3); see FASTLSQ_OPT_TENSOR_CORE */
    int32_t status;            /* as the return value of the call                  */
    double resid_norm[65];     /* ||rhs - A beta|| (incl. sqrt(mu) rows) after the  */
                               /* first solve and after each refinement step (FP64) */
} fastlsq_solve_stats;

/*
 * beta = argmin ||A beta - rhs||^2 + mu ||beta||^2 (Sec. 2.3: QR; Sec. 2.4:
 * Tikhonov with mu > 0, realised as the augmented rows sqrt(mu) I).
 *
 * A: n_rows x n_feat, dtype a_dtype, column-major with ldA (not modified; it is
 * copied into the factor's storage, FP32 for MIXED, FP64 for FP64).  rhs:
 * n_rows x nrhs (ld_rhs), beta: n_feat x nrhs (ld_beta), both double.
 * prec FP64 requires a_dtype F64.  prec MIXED refines each rhs max_refine times
 * with the FP64 residual against A_refine (double, n_rows x n_feat, ld_refine),
 * which must equal A to double precision (assemble it with dtype F64), in the
 * given refine_mode (fastlsq_refine) with max_refine steps and refine_tol (CGLS);
 * A_refine may be NULL only when max_refine is 0.
 * keep: if non-NULL, receives the factor handle (Householder reflectors, T
 * blocks, R) for fastlsq_factor_solve / fastlsq_backward; the handle keeps the
 * A_refine pointer, which must then outlive it.  stats may be NULL; if given,
 * the call synchronises the stream to fill it.
 * Requires n_rows + (mu > 0 ? n_feat : 0) >= n_feat.
 */
FASTLSQ_API int fastlsq_lstsq(fastlsq_ctx *ctx, fastlsq_prec prec,
                  const void *A, fastlsq_dtype a_dtype, int64_t ldA,
                  int64_t n_rows, int64_t n_feat, double mu,
                  const double *rhs, int32_t nrhs, int64_t ld_rhs,
                  double *beta, int64_t ld_beta,
                  const double *A_refine, int64_t ld_refine, int32_t max_refine,
                  int32_t refine_mode, double refine_tol,
                  fastlsq_factor **keep, fastlsq_solve_stats *stats);

/* Solve again with checkpointed factors for new right-hand sides (the paper's
 * matrix caching, App. G.5): beta = R^{-1} Q^T [rhs; 0], refined as in
 * fastlsq_lstsq when the factor is MIXED and was given A_refine. */
FASTLSQ_API int fastlsq_factor_solve(fastlsq_ctx *ctx, const fastlsq_factor *f,
                         const double *rhs, int32_t nrhs, int64_t ld_rhs,
                         double *beta, int64_t ld_beta, int32_t max_refine,
                         int32_t refine_mode, double refine_tol,
                         fastlsq_solve_stats *stats);

/* Copy the triangular factor R (n_feat x n_feat, upper; zeros below) of a
 * checkpointed factorisation into R_out (double, column-major, ld_r >= n_feat). */
FASTLSQ_API int fastlsq_factor_get_r(fastlsq_ctx *ctx, const fastlsq_factor *f, double *R_out,
                                     int64_t ld_r);

/* x = R^{-1} y (transpose 0) or R^{-T} y (transpose 1) in FP64 arithmetic with the
 * factor's R, by the grid-wide substitution kernel used as the Krylov
 * preconditioner.  y, x: [n_feat] double (may alias). */
FASTLSQ_API int fastlsq_factor_trsv(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *y,
                                    double *x, int32_t transpose);

/* Release a factor handle (stream-ordered). */
FASTLSQ_API int fastlsq_factor_destroy(fastlsq_factor *f);

/*
 * Adjoint of the regularised solve beta = (A^T A + mu I)^{-1} A^T rhs
 * (Sec. 2.5; Sec. 3.8: "each evaluation costs two triangular back-substitutions"),
 * with R^T R = A^T A + mu I from the checkpointed factor:
 *   v = R^{-1} R^{-T} grad_beta                      (n_feat, double, out)
 *   grad_rhs = A v                                   (n_rows, double, out; NULL to skip)
 * A_op is the FP64 operator (n_rows x n_feat, ld) used for A v; NULL uses the
 * factor's A_refine.  max_iter > 0 (either factor) computes v by preconditioned
 * CG on (A^T A + mu I) v = grad_beta with FP64 operator products (M = R^T R), up to
 * max_iter iterations or a residual reduction by tol; this needs the factor's
 * A_refine (for an FP64 factor, the operator it was factored from).  max_iter = 0
 * applies the two substitutions alone, whose relative error grows like
 * kappa(R)^2 times the factor's rounding unit.  Loss gradients with respect to a source parameter theta
 * follow as sum_i grad_rhs[i] d rhs_i / d theta (fastlsq_source_grad), and with
 * respect to operator coefficients from fastlsq_coef_grad.
 */
FASTLSQ_API int fastlsq_backward(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *grad_beta,
                     double *v, double *grad_rhs, const double *A_op, int64_t ld_op,
                     int32_t max_iter, double tol);

/*
 * dL/dtheta for the Gaussian source (problem GAUSS_SOURCE_2D):
 *   dtheta[q] = sum_i w[i] * d s(x_i; theta) / d theta_q,  x: [n][2], w = dL/df at x.
 * theta: host [n_src * 4]; dtheta: host [n_src * 4] (the call synchronises).
 */
FASTLSQ_API int fastlsq_source_grad(fastlsq_ctx *ctx, const double *x, int64_t n, const double *theta,
                        int32_t n_src, const double *w, double *dtheta);

/*
 * Gradient of the loss with respect to the coefficients of the interior operator
 * terms (PDE-coefficient parameters).  Differentiating the normal equations
 * (A^T A + mu I) beta = A^T rhs gives
 *   dL/dc_t = sum_ij (r_i v_j - (A v)_i beta_j) * scale * D^{alpha_t} phi_j(x_i)
 * with r = rhs - A beta.  Entries of each term are assembled on the fly in FP64
 * (never stored).  x: [n_rows][d] (the rows the terms act on), r, Av: [n_rows],
 * v, beta: [n_feat]; grad: host [op->n_terms] (the call synchronises).
 */
FASTLSQ_API int fastlsq_coef_grad(fastlsq_ctx *ctx, const double *x, int64_t n_rows, const fastlsq_op *op,
                      const double *W, const double *b, int64_t n_feat, double scale,
                      const double *r, const double *Av, const double *v,
                      const double *beta, double *grad);

/* One instance of the steady inverse heat-source problem (Sec. 3.8, App. G.2 in
 * steady form): -L u = s(x; theta) in the domain (interior operator from the
 * batch call), u = 0 on the boundary rows, sensors u_s = u(x_s), loss
 * L = mean_s (u_s - y_s)^2.  All pointers are DEVICE pointers. */
typedef struct {
    int64_t n_int, n_bc, n_feat, n_sens;
    const double *x_int;      /* [n_int][2]  */
    const double *x_bc;       /* [n_bc][2]   */
    const double *W;          /* [n_feat][2] */
    const double *b;          /* [n_feat]    */
    const double *sensors;    /* [n_sens][2] */
    const double *y_obs;      /* [n_sens]    */
    const double *theta;      /* [n_src * 4] evaluation point (c_x, c_y, w, a) per source */
    double *beta;             /* out [n_feat]      */
    double *loss;             /* out [1]           */
    double *dtheta;           /* out [n_src * 4]   */
} fastlsq_inverse_instance;

typedef struct {
    int32_t prec;             /* fastlsq_prec of the factorisation                    */
    int32_t refine_iters;     /* CGLS iterations of the forward solve (MIXED)         */
    double refine_tol;
    int32_t adjoint_iters;    /* PCG iterations of the adjoint solve (MIXED)          */
    double adjoint_tol;
    double mu;                /* Tikhonov parameter (rows sqrt(mu) I)                 */
    double bc_weight;         /* boundary penalty lambda                              */
} fastlsq_inverse_opts;

/*
 * Loss and gradient dL/dtheta for a batch of instances of uneven size (the
 * differentiable solve of Sec. 2.5 applied to the inverse problem of Sec. 3.8):
 * per instance, assemble the operator (FP64, plus FP32 for a MIXED factor),
 * factor it, solve for beta with the source s(x; theta), read the sensors, form
 * the loss, and run the adjoint: grad_beta = H_s^T dL/du_s,
 * v = (A^T A + mu I)^{-1} grad_beta, dL/ds = A v, dL/dtheta = sum_i (A v)_i
 * ds(x_i)/dtheta.  op is the interior operator (e.g. -Lap); n_src Gaussian
 * sources.  Queued on the context's stream without host synchronisation (the
 * whole batch can be captured in a CUDA graph once the workspace has been sized
 * by a first call).
 */
FASTLSQ_API int fastlsq_inverse_batch(fastlsq_ctx *ctx, const fastlsq_inverse_instance *inst,
                                      int32_t n_inst, const fastlsq_op *op, int32_t n_src,
                                      const fastlsq_inverse_opts *opts);

/*
 * Pre-factored batch of inverse-problem instances (Sec. 3.8: the operator is factored
 * once and every evaluation of the forward map and its gradient reuses the factor,
 * two triangular solves per evaluation; Sec. 2.5: gradients through the solve).
 *
 * fastlsq_inverse_prepare assembles each instance's FP64 operator (interior rows op,
 * boundary rows bc_weight * identity), factors [A; sqrt(mu) I] by FP64 Householder QR
 * (the factor is kept by the plan; with FASTLSQ_OPT_INVERSE_THIN_Q set, the default,
 * also Qi = the interior rows of Q [I; 0]), tabulates the sensor matrix H_s[s][j] =
 * scale sin(W_j . x_s + b_j) and records the instances' device pointers.  opts: mu > 0
 * and bc_weight are used; prec, refine and adjoint fields are ignored (the factor is
 * FP64).  The factorisations run a few at a time on worker streams of the library's
 * own, after the work already queued on the context's stream.  Limits: n_src <= 8,
 * n_sens <= 256, and a quarter of n_int + n_bc + n_feat (thin-Q plans: all of n_int)
 * plus n_feat FP64 values fitting in a CTA's shared memory, else -1 (the evaluation's
 * configuration must fit too).  Synchronises the context's stream; returns 0 and
 * *plan, or a negative status (nothing is kept).
 *
 * fastlsq_inverse_eval runs one gradient evaluation of every instance in ONE
 * persistent launch: a grid of min(n_inst, SMs * ctas_per_sm / cluster) clusters of
 * `cluster` CTAs (1, 2 or 4) of `threads` threads (256 or 512) takes instances from a
 * device-side queue, longest first (m_aug n_feat); one cluster evaluates an instance
 * entirely, its m_aug-vectors dealt over the ranks in stripes of 32 rows:
 *   y = Q^T [s(x_int; theta); 0; 0], beta = R^{-1} y[0:n], u_s = H_s beta,
 *   loss = mean (u_s - y_obs)^2, w = R^{-T} H_s^T dloss/du_s, z = Q [w; 0]
 *   (= A (A^T A + mu I)^{-1} H_s^T g), dtheta = sum_{i < n_int} z_i ds(x_i)/dtheta
 *   (thin-Q plans: y[0:n] = Qi^T s and z[0:n_int] = Qi w, the same quantities),
 * writing beta, loss and dtheta through the instances' pointers.  It reads theta and
 * y_obs at run time, allocates nothing and does not synchronise, so it can be captured
 * in a CUDA graph and replayed after the caller updates theta or y_obs in place.  No
 * cluster waits on another (the queue is one atomic counter); the ranks of a cluster
 * meet at hardware cluster barriers.  Results are deterministic for a given cluster
 * size (fixed summation orders); other cluster sizes sum in another order.  -1 for
 * other threads, cluster or ctas_per_sm values (1..4), or a shape whose shared memory
 * does not fit.
 *
 * fastlsq_inverse_plan_destroy synchronises the plan's stream and frees the factors,
 * the sensor matrices and the tables.
 */
typedef struct fastlsq_inverse_plan fastlsq_inverse_plan;
FASTLSQ_API int fastlsq_inverse_prepare(fastlsq_ctx *ctx, const fastlsq_inverse_instance *inst,
                                        int32_t n_inst, const fastlsq_op *op, int32_t n_src,
                                        const fastlsq_inverse_opts *opts, fastlsq_inverse_plan **plan);
FASTLSQ_API int fastlsq_inverse_eval(fastlsq_ctx *ctx, const fastlsq_inverse_plan *plan,
                                     int32_t threads, int32_t ctas_per_sm, int32_t cluster);
FASTLSQ_API int fastlsq_inverse_plan_destroy(fastlsq_inverse_plan *plan);

/*
 * Feature-weight and bias gradients through the exact inner solve (learnable
 * bandwidth, App. "Learnable Bandwidth via Reparameterisation", Alg. 2).  For the
 * block A_ij = row_weight * scale * sum_t coef_t D^{alpha_t} phi_j(x_i) of op (no
 * per-point terms) and the adjoint weights
 *   w_ij = r_i (c_v v_j + c_rb beta_j) + c_av (A v)_i beta_j
 * (r = rhs - A beta on these rows, v = (A^T A + mu I)^{-1} g, Av = (A v) on these rows),
 * it accumulates
 *   gW[j*d + k] += sum_i w_ij dA_ij/dW_jk,     gb[j] += sum_i w_ij dA_ij/db_j
 * with the entries' derivatives formed on the fly in FP64 from eq. cyclic (never
 * stored).  A loss that sees A only through beta with grad_beta = g takes (c_v, c_rb,
 * c_av) = (1, 0, -1); the outer loss ||A beta - rhs||^2 of Alg. 2 takes v =
 * (A^T A + mu I)^{-1} beta and (-2 mu, -2, 2 mu), or v = Av = NULL when mu = 0.  Call
 * once per row block (interior rows with the PDE operator, boundary rows with the
 * identity operator and the boundary weight); zero gW and gb first.  x: [n_rows][d];
 * W: [n_feat][d]; b, beta, v: [n_feat]; r, Av: [n_rows]; gW: [n_feat][d]; gb: [n_feat]
 * or NULL; v and Av may be NULL (their terms dropped).  All device, stream-ordered.
 */
FASTLSQ_API int fastlsq_weight_grad(fastlsq_ctx *ctx, const double *x, int64_t n_rows,
                                    const fastlsq_op *op, double row_weight, const double *W,
                                    const double *b, int64_t n_feat, double scale,
                                    const double *r, const double *beta, const double *v,
                                    const double *Av, double c_v, double c_rb, double c_av,
                                    double *gW, double *gb);

/*
 * Contraction of a feature-weight gradient with the frozen base weights W_hat:
 *   out[a*d + c] = sum_j gW[j][a] W_hat[j][c],     out[d*d] = sum_a out[a*d + a],
 * so that for W_j = L W_hat_j (eq. reparam_cholesky) dL/dL_ac = out[a*d + c] (take
 * the lower triangle) and for W = sigma W_hat (eq. reparam_scalar) dL/dsigma =
 * out[d*d].  gW, W_hat: [n_feat][d]; out: [d*d + 1]; all device.
 */
FASTLSQ_API int fastlsq_bandwidth_grad(fastlsq_ctx *ctx, const double *gW, const double *W_hat,
                                       int64_t n_feat, int32_t d, double *out);

/*
 * r = rhs - A beta in FP64 (eq. linear_system's residual), A: m x n column-major
 * (ld >= m), beta: [n], rhs, r: [m]; all device.
 */
FASTLSQ_API int fastlsq_residual(fastlsq_ctx *ctx, const double *A, int64_t ld, int64_t m,
                                 int64_t n, const double *beta, const double *rhs, double *r);

/* Nonlinearities N(u) of the Newton problems (Sec. 3.3): nl_lam e^u, nl_lam u^3, or the
 * Burgers advection term nl_lam u du/dx_0 (derivative along the first coordinate). */
typedef enum { FASTLSQ_NL_NONE = 0, FASTLSQ_NL_EXP = 1, FASTLSQ_NL_CUBIC = 2,
               FASTLSQ_NL_BURGERS = 3 } fastlsq_nl;

typedef struct {
    int32_t d;
    int64_t n_int, n_bc;
    const double *x_int;      /* [n_int][d] */
    const double *x_bc;       /* [n_bc][d]  */
    fastlsq_op op;            /* interior linear operator L (no per-point terms) */
    int32_t nl_kind;          /* fastlsq_nl: N(u) = nl_lam e^u, nl_lam u^3 or     */
                              /* nl_lam u u_{x_0}                                */
    double nl_lam;
    double bc_weight;         /* boundary rows bc_weight * (u - g) (Dirichlet)   */
    const double *f;          /* [n_int] */
    const double *g;          /* [n_bc]  */
} fastlsq_newton_problem;

typedef struct {
    int32_t max_iter;         /* <= 64                                           */
    double tol;               /* stop when ||a J_u delta|| / ||u|| <= tol        */
    double mu;                /* Tikhonov parameter of each step                 */
    double armijo_c;          /* accept a when ||R(beta+a delta)||^2 <= (1-2ca)||R||^2 */
    int32_t max_halvings;     /* backtracking halvings before giving up          */
    int32_t prec;             /* fastlsq_prec of each step's solve               */
    int32_t max_refine;       /* CGLS refinement iterations per step (MIXED)     */
    double refine_tol;        /* CGLS tolerance per step (0: 1e-10)              */
} fastlsq_newton_opts;

typedef struct {
    int32_t iters;
    int32_t status;
    double res_norm[65];      /* ||R|| before each iteration and after the last  */
    double step_rel[64];      /* ||a J_u delta|| / ||u|| per iteration            */
    double alpha[64];         /* accepted step length per iteration              */
} fastlsq_newton_stats;

/*
 * Newton-Raphson for L[u] + N[u] = f with Dirichlet rows (Sec. 2.4, eq. newton):
 * R_i = L[u](x_i) + N(u_i) - f_i (interior), bc_weight (u_i - g_i) (boundary);
 * J_ij = L[phi_j](x_i) + N'(u_i) phi_j(x_i) reassembled on the GPU every
 * iteration (Burgers: + nl_lam u_{x_0}(x_i) phi_j(x_i) + nl_lam u(x_i) d(phi_j)/dx_0(x_i),
 * the second a per-point coefficient on a first-derivative feature); delta = argmin ||J delta + R||^2 + mu ||delta||^2; Armijo
 * backtracking on ||R||; solution-level stopping test.  beta_inout: [n_feat]
 * (start value in, solution out; a warm start from the linear part is the
 * caller's choice).  The residuals and the refinement operator are FP64.  The
 * call synchronises once per iteration to take the line-search decisions and
 * fills stats (may be NULL).  Returns 0 converged, 1 max_iter, 2 line search
 * failed, or an error.
 */
FASTLSQ_API int fastlsq_newton(fastlsq_ctx *ctx, const fastlsq_newton_problem *prob,
                   const double *W, const double *b, int64_t n_feat, double scale,
                   const fastlsq_newton_opts *opts, double *beta_inout,
                   fastlsq_newton_stats *stats);

/*
 * Newton with continuation (homotopy, Sec. 2.4, used for steady Burgers): n_stages
 * fastlsq_newton solves in turn, stage k with the interior operator's term
 * coefficients replaced by stage_coef[k * prob->op.n_terms + t] (e.g. the viscosity
 * term -nu D^2 with nu = 1.0, 0.5, 0.2, 0.1), each stage starting from the previous
 * stage's beta (beta_inout: start value in, last stage's solution out).  The other
 * fields of prob (nonlinearity, data, weights) stay fixed.  stats: host
 * [n_stages] (may be NULL).  Returns the last stage's status (0 converged,
 * 1 max_iter, 2 line search failed); an error of any stage is returned at once.
 * A stage whose status is 2 ends the continuation.
 */
FASTLSQ_API int fastlsq_newton_continuation(fastlsq_ctx *ctx, const fastlsq_newton_problem *prob,
                   const double *W, const double *b, int64_t n_feat, double scale,
                   const fastlsq_newton_opts *opts, int32_t n_stages,
                   const double *stage_coef, double *beta_inout,
                   fastlsq_newton_stats *stats);

/*
 * Self-test of the bounded device waits (failure detection; the paper has no
 * counterpart).  Launches, on the context's stream, a kernel whose wait never
 * completes: which = 0, an mbarrier wait like those of the tensor-core kernels on a
 * barrier nobody arrives on (one CTA); which = 1, the grid barrier of the cooperative
 * kernels with one of its two CTAs leaving without arriving.  After budget_cycles SM
 * clock cycles (0 .. 4e9; the library's own waits use about 2e9, a second) the waiting
 * thread raises the context's device error flag and the kernel returns: the next
 * fastlsq_sync returns FASTLSQ_ERR_TIMEOUT, clears the flag and resets the grid
 * barrier, and the context stays usable.  Returns 0 once queued, -1 for other
 * arguments, -3 if the launch fails.
 */
FASTLSQ_API int fastlsq_selftest_wait(fastlsq_ctx *ctx, int32_t which, int64_t budget_cycles);

/* Context options for fastlsq_set_option. */
typedef enum {
    FASTLSQ_OPT_TENSOR_CORE = 0,  /* trailing updates of the MIXED (FP32) factorisation.
                                      1 (default): two-level blocking: outer blocks of 128
                                      columns, each factored as panels of width 32 (16 for
                                      panels taller than the register panels hold) with
                                      SIMT FP32 updates inside the block, then one update
                                      of every column right of the block on tcgen05 with
                                      K = 128, operands split into three bf16 parts (six
                                      products: FP32-level accuracy), FP32 accumulation;
                                      used for factors refined classically and by CGLS.
                                      2: panel by panel on tcgen05 with TF32x3 products
                                      (2^-22 relative, operands by TMA) for panel width 32
                                      in factors refined classically (CGLS-refined factors
                                      then use the SIMT update).  0: SIMT FP32 panel by
                                      panel everywhere. */
    FASTLSQ_OPT_REGISTER_PANEL = 1, /* 1 (default): FP32 panels of width 32 factor with the
                                      slice in registers where rows per warp <= 24;
                                      0: the shared-memory panel kernel everywhere */
    FASTLSQ_OPT_LOOKAHEAD = 2,     /* 1 (default): panel p+1 is factored on the caller's
                                      stream while the rest of panel p's trailing update runs
                                      on a second, low-priority stream of the context (joined
                                      back into the caller's stream before the next panel's
                                      update); in the two-level factor the outer-block
                                      update pass also does the next block's columns first
                                      and the rest on a third stream beside that block's
                                      panels; 0: everything on the caller's stream, one
                                      update pass per panel (faster when several
                                      independent solves run on other streams and fill
                                      the SMs beside each panel) */
    FASTLSQ_OPT_TRSV_FP32 = 3,     /* 1 (default): the triangular solves of classical
                                      refinement (MIXED) substitute in FP32 arithmetic
                                      (backward stable like the FP32 factor); 0: FP64
                                      arithmetic.  CGLS and the adjoint: see
                                      FASTLSQ_OPT_KRYLOV_DF. */
    FASTLSQ_OPT_FUSED_LOOKAHEAD = 4,/* 1 (default): with look-ahead, the register panel
                                      applies the previous panel's update to its own columns
                                      in its prologue (no separate kernels for it) where its
                                      shared memory allows; 0: separate update kernels */
    FASTLSQ_OPT_ROW_PANEL = 5,      /* 1 (default): the register panel keeps one or two
                                      panel rows per thread (updates without shuffles),
                                      where the panel has at most 768 rows per CTA; 0: one
                                      column per lane (32 rows per thread at most) */
    FASTLSQ_OPT_SPLIT_ROWS = 6,     /* least rows per split of the SIMT trailing updates'
                                      Y pass (a multiple of 32, 32 .. 1048576; default 256).
                                      Small splits give one solve the shortest latency;
                                      larger ones launch fewer CTAs per update, leaving
                                      more of the GPU to other solves running beside it */
    FASTLSQ_OPT_INVERSE_THIN_Q = 7, /* 1 (default): fastlsq_inverse_prepare also forms each
                                      instance's thin Q restricted to its interior rows,
                                      Qi = (Q [I; 0])[0:n_int] (n_int x n FP64, about the
                                      factorisation's FP64 work again), and the evaluations
                                      use Qi^T s and Qi w: 2 n_int n FMAs per instance
                                      instead of 4 m_aug n with the reflectors; 0: the
                                      plan keeps the reflectors only (faster setup, less
                                      memory). Read when a plan is prepared. */
    FASTLSQ_OPT_FP64_ASSEMBLY_CTAS = 8, /* FP64 operator assembly launch: 0 (default) one CTA
                                      of 256 threads per 128 x 64 tile of entries; k = 1..8
                                      a persistent grid of k CTAs per SM looping over the
                                      tiles (a smaller footprint beside kernels of other
                                      streams).  The entries are the same either way. */
    FASTLSQ_OPT_KRYLOV_DF = 9       /* 1 (default): the preconditioner solves R^{-1}, R^{-T}
                                      of CGLS refinement and of the PCG adjoint with an FP32
                                      factor run in double-float arithmetic (pairs of FP32
                                      values, about 48 bits) on the FP32 pipes; 0: FP64
                                      arithmetic.  The Krylov vectors, products and
                                      residuals stay FP64, and fastlsq_factor_trsv is always
                                      FP64. */
} fastlsq_option;

/* Set a context option (see fastlsq_option).  Returns 0 or -1 for an unknown option. */
FASTLSQ_API int fastlsq_set_option(fastlsq_ctx *ctx, int option, int value);

/* Kernel classes for profiling (launch counts are always kept; device times are
 * recorded with CUDA events around each launch only while profiling is on). */
typedef enum {
    FASTLSQ_K_PREFACTOR = 0,   /* column prefactors P, Q                          */
    FASTLSQ_K_ASSEMBLE_F32,    /* operator assembly, FP32 (SFU)                   */
    FASTLSQ_K_ASSEMBLE_F64,    /* operator assembly, FP64                         */
    FASTLSQ_K_RHS,             /* right-hand sides                                */
    FASTLSQ_K_EVAL,            /* u at points                                     */
    FASTLSQ_K_COPY_IN,         /* matrix into factor storage (+ Tikhonov rows)    */
    FASTLSQ_K_PANEL,           /* Householder panel (cluster)                     */
    FASTLSQ_K_TRAIL_SIMT,      /* trailing update, SIMT                           */
    FASTLSQ_K_TRAIL_TC,        /* trailing update, tcgen05 TF32x3                 */
    FASTLSQ_K_APPLY_Q,         /* Q^T y / Q y                                     */
    FASTLSQ_K_TRSV,            /* triangular solves                               */
    FASTLSQ_K_RESIDUAL,        /* FP64 residual / matvec                          */
    FASTLSQ_K_VECTOR,          /* small vector kernels                            */
    FASTLSQ_K_NEWTON,          /* Newton pointwise kernels                        */
    FASTLSQ_K_ADJOINT,         /* adjoint contractions                            */
    FASTLSQ_K_KRYLOV,          /* Krylov refinement (FP64 products, scalars)      */
    FASTLSQ_K_BLOCK_PREP,      /* outer-block update: operand images of V and Z   */
    FASTLSQ_K_BLOCK_Y,         /* outer-block update: Y = V^T [V | C], tcgen05    */
    FASTLSQ_K_BLOCK_U,         /* outer-block update: C -= V Z, tcgen05           */
    FASTLSQ_K_COUNT
} fastlsq_kernel;

/* Record per-launch CUDA-event times on the context's stream for the kernel
 * classes whose bit (1 << fastlsq_kernel) is set in `mask` (0 stops recording,
 * -1 records every class); any call clears all counters.  Must be 0 while the
 * stream is being captured into a CUDA graph. */
FASTLSQ_API int fastlsq_profile_enable(fastlsq_ctx *ctx, int mask);
/* Launches of kernel class `kernel` since the last reset, and (if profiling was
 * on) their summed device time in milliseconds.  Synchronises the stream. */
FASTLSQ_API int fastlsq_profile_read(fastlsq_ctx *ctx, int kernel, int64_t *launches,
                                     double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* FASTLSQ_H */

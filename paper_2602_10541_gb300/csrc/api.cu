// C ABI entry points of libfastlsq (declared in include/fastlsq.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "common.cuh"
#include "qr.cuh"

int fl_launch_eval(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d, const double *W,
                   const double *b, int64_t n_feat, double scale, const double *beta, double *u);
int fl_launch_eval_op(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d, const double *W,
                      const double *b, int64_t n_feat, const double *pref, const double *beta, double *u);
int fl_launch_eval_noalloc(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d, const double *W,
                           const double *b, int64_t n_feat, double scale, const double *beta, double *u);
cudaError_t fl_eval_static_lookup(double **out);
int fl_launch_eval_adjoint(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int d,
                           const double *W, const double *b, int64_t n_feat, double scale,
                           const double *g, double *grad);
int fl_launch_rhs(fastlsq_ctx *ctx, int problem, int kind, const double *params, int n_params,
                  const double *x, int64_t n, int d, double weight, double *out);
int fl_launch_source_grad(fastlsq_ctx *ctx, const double *x, int64_t n, const double *theta,
                          int n_src, const double *w, double *dtheta_host);
int fl_launch_coef_grad(fastlsq_ctx *ctx, const double *x, int64_t n_rows, const fl_op_params &op,
                        const double *W, const double *b, int64_t n_feat, double scale,
                        const double *r, const double *Av, const double *v, const double *beta,
                        double *grad_host);

// ---------------------------------------------------------------------------
// errors and workspace
// ---------------------------------------------------------------------------
int fl_fail(fastlsq_ctx *ctx, int code, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return code;
}

int fl_cuda(fastlsq_ctx *ctx, cudaError_t e, const char *what)
{
    int code = (e == cudaErrorMemoryAllocation) ? FASTLSQ_ERR_NOMEM : FASTLSQ_ERR_CUDA;
    return fl_fail(ctx, code, "%s: %s", what, cudaGetErrorString(e));
}

void *fl_ws(fastlsq_ctx *ctx, int slot, size_t bytes)
{
    fl_buffer &b = ctx->ws[slot];
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return b.ptr;
    // stream-ordered: kernels already queued on the old buffer finish before it is freed
    if (b.ptr) cudaFreeAsync(b.ptr, ctx->stream);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 4;
    cudaError_t e = cudaMallocAsync(&b.ptr, want, ctx->stream);
    if (e != cudaSuccess) {
        fl_cuda(ctx, e, "workspace allocation");
        b.ptr = nullptr;
        return nullptr;
    }
    b.bytes = want;
    return b.ptr;
}

static void *fl_alloc(fastlsq_ctx *ctx, size_t bytes, int *rc)
{
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes ? bytes : 16, ctx->stream);
    if (e != cudaSuccess) {
        *rc = fl_cuda(ctx, e, "allocation");
        return nullptr;
    }
    return p;
}

int fl_pack_op(fastlsq_ctx *ctx, const fastlsq_op *op, fl_op_params *out)
{
    if (!op) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "operator is NULL");
    if (op->d < 1 || op->d > FL_MAX_D)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "d = %d outside 1..%d", op->d, FL_MAX_D);
    if (op->n_terms < 0 || op->n_terms > FL_MAX_TERMS)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "n_terms = %d outside 0..%d", op->n_terms, FL_MAX_TERMS);
    if (op->n_pp < 0 || op->n_pp > FL_MAX_PP)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "n_pp = %d outside 0..%d", op->n_pp, FL_MAX_PP);
    if (op->n_terms > 0 && (!op->alpha || !op->coef))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "operator terms missing");
    memset(out, 0, sizeof(*out));
    out->d = op->d;
    out->n_terms = op->n_terms;
    for (int t = 0; t < op->n_terms; ++t) {
        out->coef[t] = op->coef[t];
        for (int k = 0; k < op->d; ++k) {
            int a = op->alpha[t * op->d + k];
            if (a < 0 || a > 16) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "alpha entry %d", a);
            out->alpha[t][k] = a;
        }
    }
    out->n_pp = op->n_pp;
    for (int q = 0; q < op->n_pp; ++q) {
        if (!op->pp_alpha || !op->pp_coef || !op->pp_coef[q])
            return fl_fail(ctx, FASTLSQ_ERR_INVALID, "per-point term %d missing", q);
        out->pp_coef[q] = op->pp_coef[q];
        for (int k = 0; k < op->d; ++k) {
            int a = op->pp_alpha[q * op->d + k];
            if (a < 0 || a > 16) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "alpha entry %d", a);
            out->pp_alpha[q][k] = a;
        }
    }
    return 0;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
static float trunc_mantissa(float v, int keep_bits)
{
    uint32_t u;
    memcpy(&u, &v, 4);
    u &= ~((1u << (23 - keep_bits)) - 1u);
    memcpy(&v, &u, 4);
    return v;
}

extern "C" int fastlsq_create(fastlsq_ctx **out, int device, void *stream)
{
    if (!out) return FASTLSQ_ERR_INVALID;
    *out = nullptr;
    fastlsq_ctx *ctx = new (std::nothrow) fastlsq_ctx();
    if (!ctx) return FASTLSQ_ERR_NOMEM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream);
    // the address of fastlsq_eval_noalloc's fixed scratch in this device's context (this
    // also loads the library's device code now, so the array is committed here and a
    // context created after a device reset gets the array's new address)
    if (e == cudaSuccess) e = fl_eval_static_lookup(&ctx->eval_static);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_grid_bar, 64);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_grid_bar, 0, 64, ctx->stream);
    if (e == cudaSuccess) {
        // keep freed stream-ordered memory cached in the pool (no per-call OS round trips)
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    }
    if (e == cudaSuccess) {
        // low-priority stream for the trailing updates that run beside a look-ahead panel
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->aux_stream, cudaStreamNonBlocking, lo);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->aux2_stream, cudaStreamNonBlocking, lo);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork2, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        int rc = (e == cudaErrorMemoryAllocation) ? FASTLSQ_ERR_NOMEM : FASTLSQ_ERR_CUDA;
        if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
        if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
        if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
        if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
        if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
        if (ctx->aux2_stream) cudaStreamDestroy(ctx->aux2_stream);
        if (ctx->d_flag) cudaFree(ctx->d_flag);
        if (ctx->d_grid_bar) cudaFree(ctx->d_grid_bar);
        delete ctx;
        return rc;
    }
    // Cody-Waite split of 2 pi: c1, c2 with 12 significant bits each (so q * c_i is
    // exact for |q| < 2^12), c3 the float rounding of the remainder
    const double twopi = 6.283185307179586476925286766559;
    float c1 = trunc_mantissa((float)twopi, 11);
    float c2 = trunc_mantissa((float)(twopi - (double)c1), 11);
    float c3 = (float)(twopi - (double)c1 - (double)c2);
    ctx->cw2pi[0] = c1;
    ctx->cw2pi[1] = c2;
    ctx->cw2pi[2] = c3;
    *out = ctx;
    return 0;
}

fl_prof_scope::fl_prof_scope(fastlsq_ctx *c, int kid, int n_launches) : ctx(c), id(kid)
{
    ctx->prof.launches[id] += n_launches;
    if (!ctx->prof.enabled || !((ctx->prof.mask >> id) & 1u)) return;
    auto &pool = ctx->prof.ev[id];
    size_t u = ctx->prof.used[id];
    while (pool.size() < u + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        pool.push_back(e);
    }
    cudaEventRecord(pool[u], ctx->stream);
    end = pool[u + 1];
    ctx->prof.used[id] = u + 2;
}

fl_prof_scope::~fl_prof_scope()
{
    if (end) cudaEventRecord(end, ctx->stream);
}

static void prof_collect(fastlsq_ctx *ctx)
{
    cudaStreamSynchronize(ctx->stream);
    if (ctx->aux_stream) cudaStreamSynchronize(ctx->aux_stream);
    if (ctx->aux2_stream) cudaStreamSynchronize(ctx->aux2_stream);
    for (int k = 0; k < FASTLSQ_K_COUNT; ++k) {
        for (size_t i = 0; i + 1 < ctx->prof.used[k]; i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ctx->prof.ev[k][i], ctx->prof.ev[k][i + 1]) == cudaSuccess)
                ctx->prof.ms[k] += ms;
        }
        ctx->prof.used[k] = 0;
    }
}

extern "C" int fastlsq_profile_enable(fastlsq_ctx *ctx, int mask)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (ctx->prof.enabled) prof_collect(ctx);
    for (int k = 0; k < FASTLSQ_K_COUNT; ++k) {
        ctx->prof.launches[k] = 0;
        ctx->prof.ms[k] = 0.0;
        ctx->prof.used[k] = 0;
    }
    ctx->prof.mask = (unsigned)mask;
    ctx->prof.enabled = mask != 0;
    return 0;
}

extern "C" int fastlsq_profile_read(fastlsq_ctx *ctx, int kernel, int64_t *launches, double *total_ms)
{
    if (!ctx || kernel < 0 || kernel >= FASTLSQ_K_COUNT) return FASTLSQ_ERR_INVALID;
    if (ctx->prof.enabled) prof_collect(ctx);
    else cudaStreamSynchronize(ctx->stream);
    if (launches) *launches = ctx->prof.launches[kernel];
    if (total_ms) *total_ms = ctx->prof.ms[kernel];
    return 0;
}

extern "C" int fastlsq_destroy(fastlsq_ctx *ctx)
{
    if (!ctx) return 0;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->aux_stream) cudaStreamSynchronize(ctx->aux_stream);
    if (ctx->aux2_stream) cudaStreamSynchronize(ctx->aux2_stream);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
    if (ctx->ev_join2) cudaEventDestroy(ctx->ev_join2);
    if (ctx->aux2_stream) cudaStreamDestroy(ctx->aux2_stream);
    for (int k = 0; k < FASTLSQ_K_COUNT; ++k)
        for (cudaEvent_t e : ctx->prof.ev[k]) cudaEventDestroy(e);
    for (int s = 0; s < FL_WS_COUNT; ++s)
        if (ctx->ws[s].ptr) cudaFree(ctx->ws[s].ptr);
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    if (ctx->d_grid_bar) cudaFree(ctx->d_grid_bar);
    delete ctx;
    return 0;
}

extern "C" int fastlsq_set_stream(fastlsq_ctx *ctx, void *stream)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    ctx->stream = (cudaStream_t)stream;
    return 0;
}

extern "C" int fastlsq_set_refine_event(fastlsq_ctx *ctx, void *event)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    ctx->refine_event = (cudaEvent_t)event;
    return 0;
}

// the stream waits for the caller's event before the first read of A_refine
static int wait_refine(fastlsq_ctx *ctx)
{
    if (!ctx->refine_event) return 0;
    cudaError_t e = cudaStreamWaitEvent(ctx->stream, ctx->refine_event, 0);
    return e == cudaSuccess ? 0 : fl_cuda(ctx, e, "wait for the FP64 operator");
}

extern "C" int fastlsq_set_option(fastlsq_ctx *ctx, int option, int value)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (option == FASTLSQ_OPT_TENSOR_CORE) {
        if (value < FL_TC_SIMT || value > FL_TC_PANEL)
            return fl_fail(ctx, FASTLSQ_ERR_INVALID, "tensor-core mode %d outside 0..2", value);
        ctx->use_tensor_core = value;
        return 0;
    }
    if (option == FASTLSQ_OPT_REGISTER_PANEL) {
        ctx->panel_reg = value ? 1 : 0;
        return 0;
    }
    if (option == FASTLSQ_OPT_LOOKAHEAD) {
        ctx->lookahead = value ? 1 : 0;
        return 0;
    }
    if (option == FASTLSQ_OPT_ROW_PANEL) {
        ctx->row_panel = value ? 1 : 0;
        return 0;
    }
    if (option == FASTLSQ_OPT_FUSED_LOOKAHEAD) {
        ctx->fuse_next = value ? 1 : 0;
        return 0;
    }
    if (option == FASTLSQ_OPT_TRSV_FP32) {
        ctx->trsv32 = value ? 1 : 0;
        return 0;
    }
    if (option == FASTLSQ_OPT_KRYLOV_DF) {
        ctx->krylov_df = value ? 1 : 0;
        return 0;
    }
    if (option == FASTLSQ_OPT_FP64_ASSEMBLY_CTAS) {
        if (value < 0 || value > 8)
            return fl_fail(ctx, FASTLSQ_ERR_INVALID, "FP64 assembly CTAs per SM %d outside 0..8", value);
        ctx->asm64_ctas_per_sm = value;
        return 0;
    }
    if (option == FASTLSQ_OPT_INVERSE_THIN_Q) {
        ctx->inverse_thin_q = value ? 1 : 0;
        return 0;
    }
    if (option == FASTLSQ_OPT_SPLIT_ROWS) {
        if (value < 32 || value > (1 << 20) || value % 32 != 0)
            return fl_fail(ctx, FASTLSQ_ERR_INVALID, "split rows %d: a multiple of 32 in 32 .. 1048576", value);
        ctx->split_rows = value;
        return 0;
    }
    return fl_fail(ctx, FASTLSQ_ERR_INVALID, "unknown option %d", option);
}

extern "C" const char *fastlsq_last_error(const fastlsq_ctx *ctx)
{
    return ctx ? ctx->last_error.c_str() : "null context";
}

extern "C" int fastlsq_sync(fastlsq_ctx *ctx)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "sync");
    if (flag) {
        cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream);
        // a barrier that timed out may have left arrivals counted: start it afresh
        if (flag == FL_DEVERR_TIMEOUT) cudaMemsetAsync(ctx->d_grid_bar, 0, 64, ctx->stream);
        if (flag == FL_DEVERR_NONFINITE) return fl_fail(ctx, FASTLSQ_ERR_NONFINITE, "non-finite value on the device");
        if (flag == FL_DEVERR_TIMEOUT) return fl_fail(ctx, FASTLSQ_ERR_TIMEOUT, "device-side wait timed out");
        return fl_fail(ctx, FASTLSQ_ERR_CUDA, "device error flag %d", flag);
    }
    return 0;
}

// ---------------------------------------------------------------------------
// assembly, rhs, evaluation
// ---------------------------------------------------------------------------
extern "C" int fastlsq_assemble(fastlsq_ctx *ctx, fastlsq_dtype dtype, const double *x,
                                int64_t n_rows, const fastlsq_op *op, double row_weight,
                                const double *W, const double *b, int64_t n_feat, double scale,
                                void *A, int64_t ldA, int64_t row_offset)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    fl_op_params p;
    FL_TRY(fl_pack_op(ctx, op, &p));
    if (n_rows < 0 || n_feat < 0 || n_feat > FL_MAX_FEAT || row_offset < 0)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "bad sizes (n_rows %lld, n_feat %lld)",
                       (long long)n_rows, (long long)n_feat);
    if (ldA < row_offset + n_rows) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "ldA < row_offset + n_rows");
    if (n_rows == 0 || n_feat == 0) return 0;
    if (!x || !W || !b || !A) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "null array");
    if (dtype != FASTLSQ_F32 && dtype != FASTLSQ_F64) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "dtype");
    double *pref = (double *)fl_ws(ctx, FL_WS_PREFACTOR, sizeof(double) * (2 + FL_MAX_PP) * n_feat);
    if (!pref) return FASTLSQ_ERR_NOMEM;
    FL_TRY(fl_prefactors(ctx, p, W, n_feat, scale, row_weight, pref));
    if (dtype == FASTLSQ_F32)
        return fl_launch_assemble_f32(ctx, p, x, n_rows, W, b, n_feat, pref, (float *)A, ldA,
                                      row_offset, row_weight);
    return fl_launch_assemble_f64(ctx, p, x, n_rows, W, b, n_feat, pref, (double *)A, ldA,
                                  row_offset, row_weight);
}

extern "C" int fastlsq_eval_op(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                               const fastlsq_op *op, const double *W, const double *b, int64_t n_feat,
                               double scale, const double *beta, double *u)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    fl_op_params p;
    FL_TRY(fl_pack_op(ctx, op, &p));
    if (p.n_pp != 0) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval_op: per-point coefficients are not allowed");
    if (n_eval < 0 || n_feat < 1 || n_feat > FL_MAX_FEAT || d != p.d)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval_op: bad sizes");
    if (n_eval == 0) return 0;
    if (!x || !W || !b || !beta || !u) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval_op: null array");
    double *pref = (double *)fl_ws(ctx, FL_WS_PREFACTOR, sizeof(double) * (2 + FL_MAX_PP) * n_feat);
    if (!pref) return FASTLSQ_ERR_NOMEM;
    FL_TRY(fl_prefactors(ctx, p, W, n_feat, scale, 1.0, pref));
    return fl_launch_eval_op(ctx, x, n_eval, d, W, b, n_feat, pref, beta, u);
}

extern "C" int fastlsq_rhs(fastlsq_ctx *ctx, fastlsq_problem problem, fastlsq_rhs_kind kind,
                           const double *params, int32_t n_params, const double *x, int64_t n,
                           int32_t d, double weight, double *out)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (n < 0 || d < 1 || d > FL_MAX_D || n_params < 0 || (n_params > 0 && !params))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: bad arguments");
    if (problem < FASTLSQ_PROBLEM_POISSON_1D || problem > FASTLSQ_PROBLEM_VARCOEF_2D)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: unknown problem %d", (int)problem);
    if (kind < FASTLSQ_RHS_SOURCE || kind >= FASTLSQ_RHS_COEF_GRAD + d)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: kind %d", (int)kind);
    if (kind >= FASTLSQ_RHS_COEF && problem != FASTLSQ_PROBLEM_VARCOEF_2D)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: problem %d has no variable coefficient", (int)problem);
    if (problem == FASTLSQ_PROBLEM_VARCOEF_2D && (n_params < 1 || d != 2))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: problem 10 needs d = 2 and params[0] = a");
    if ((problem == FASTLSQ_PROBLEM_ALLEN_CAHN_1D || problem == FASTLSQ_PROBLEM_BURGERS_1D) &&
        kind == FASTLSQ_RHS_EXACT && (n_params < 1 || !(params[0] > 0)))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: problem %d needs params[0] > 0", (int)problem);
    if (kind == FASTLSQ_RHS_SOURCE &&
        ((problem == FASTLSQ_PROBLEM_NLPOISSON_2D && n_params < 1) ||
         (problem == FASTLSQ_PROBLEM_NLHELMHOLTZ_2D && n_params < 2) ||
         (problem == FASTLSQ_PROBLEM_HELMHOLTZ_2D && n_params < 1)))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: problem %d needs more parameters", (int)problem);
    if (n == 0) return 0;
    if (!x || !out) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "rhs: null array");
    return fl_launch_rhs(ctx, problem, kind, params, n_params, x, n, d, weight, out);
}

extern "C" int fastlsq_eval(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                            const double *W, const double *b, int64_t n_feat, double scale,
                            const double *beta, double *u)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (n_eval < 0 || n_feat < 1 || n_feat > FL_MAX_FEAT || d < 1 || d > FL_MAX_D)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval: bad sizes");
    if (n_eval == 0) return 0;
    if (!x || !W || !b || !beta || !u) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval: null array");
    return fl_launch_eval(ctx, x, n_eval, d, W, b, n_feat, scale, beta, u);
}

extern "C" int fastlsq_eval_noalloc(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                                    const double *W, const double *b, int64_t n_feat, double scale,
                                    const double *beta, double *u)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (n_eval < 0 || n_feat < 1 || n_feat > FL_MAX_FEAT || d < 1 || d > FL_MAX_D)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval_noalloc: bad sizes");
    if (n_eval == 0) return 0;
    if (!x || !W || !b || !beta || !u) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval_noalloc: null array");
    return fl_launch_eval_noalloc(ctx, x, n_eval, d, W, b, n_feat, scale, beta, u);
}

extern "C" int fastlsq_eval_adjoint(fastlsq_ctx *ctx, const double *x, int64_t n_eval, int32_t d,
                                    const double *W, const double *b, int64_t n_feat, double scale,
                                    const double *g, double *grad_beta)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (n_eval < 0 || n_feat < 1 || d < 1 || d > FL_MAX_D)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval_adjoint: bad sizes");
    if (!x || !W || !b || !g || !grad_beta)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "eval_adjoint: null array");
    return fl_launch_eval_adjoint(ctx, x, n_eval, d, W, b, n_feat, scale, g, grad_beta);
}

// ---------------------------------------------------------------------------
// least squares
// ---------------------------------------------------------------------------
static void factor_free(fastlsq_factor *f)
{
    if (!f) return;
    cudaStream_t s = f->stream;
    if (f->F) cudaFreeAsync(f->F, s);
    if (f->tau) cudaFreeAsync(f->tau, s);
    if (f->T) cudaFreeAsync(f->T, s);
    if (f->Tb) cudaFreeAsync(f->Tb, s);
    delete f;
}

// Solve with the factors for right-hand side r: the transformed rhs Q^T b is
// either already in column n + r of F (from_factor) or computed from rhs64.
template <typename T>
static int solve_one(fastlsq_ctx *ctx, const fastlsq_factor *f, int nrhs_in_F, int r,
                     const double *rhs64, double *beta64, int max_refine, int mode, double tol,
                     double *norms_dev)
{
    const int64_t n = f->n, m = f->m, m_aug = f->m_aug;
    const T *F = (const T *)f->F;
    T *y = (T *)fl_ws(ctx, FL_WS_VEC0, sizeof(T) * m_aug);
    double *v64 = (double *)fl_ws(ctx, FL_WS_SOLVE64, sizeof(double) * 3 * n + 64);
    if (!y || !v64) return FASTLSQ_ERR_NOMEM;
    double *y64 = v64, *dx64 = v64 + n, *work = v64 + 2 * n;
    if (r < nrhs_in_F) {
        FL_TRY(fl_extract_rhs<T>(ctx, F, f->ld, n, r, y));
    } else {
        FL_TRY(fl_from_f64<T>(ctx, rhs64, m, m_aug, y));
        FL_TRY(fl_apply_q<T>(ctx, F, f->ld, m_aug, n, f->nb, (const T *)f->T, y, 1,
                             f->has_tb ? (const float *)f->Tb : nullptr));
    }
    FL_TRY(fl_to_f64<T>(ctx, y, n, y64, 0));
    // FP32 substitution (backward stable, like the FP32 factor itself) is an option for
    // classical refinement; CGLS needs R^{-1} as a fixed linear operator: FP64
    const int a32 = (mode == FASTLSQ_REFINE_CLASSICAL && ctx->trsv32) ? FL_ARITH_F32 : 0;
    FL_TRY(fl_trsv_grid<T>(ctx, F, f->ld, n, y64, beta64, work, 0, nullptr, a32));
    if ((max_refine > 0 || norms_dev) && f->A_refine) FL_TRY(wait_refine(ctx));
    if (mode == FASTLSQ_REFINE_CGLS) {
        if (max_refine > 0) return fl_refine_cgls(ctx, f, rhs64, beta64, max_refine, tol, norms_dev);
        return 0;
    }
    // classical iterative refinement: FP64 residual, correction R^{-1} Q^T r with the
    // factors (Q^T in the factor's type, R^{-1} in FP64)
    for (int it = 0; it < max_refine; ++it) {
        FL_TRY(fl_residual<T>(ctx, f->A_refine, f->ld_refine, m, n, f->mu, m_aug, rhs64, beta64, y,
                              norms_dev ? norms_dev + it : nullptr));
        FL_TRY(fl_apply_q<T>(ctx, F, f->ld, m_aug, n, f->nb, (const T *)f->T, y, 1,
                             f->has_tb ? (const float *)f->Tb : nullptr));
        FL_TRY(fl_to_f64<T>(ctx, y, n, y64, 0));
        FL_TRY(fl_trsv_grid<T>(ctx, F, f->ld, n, y64, dx64, work, 0, nullptr, a32));
        FL_TRY(fl_to_f64<double>(ctx, dx64, n, beta64, 1));
    }
    if (norms_dev && f->A_refine) {
        FL_TRY(fl_residual<T>(ctx, f->A_refine, f->ld_refine, m, n, f->mu, m_aug, rhs64, beta64, y,
                              norms_dev + max_refine));
    }
    return 0;
}

static int solve_all(fastlsq_ctx *ctx, const fastlsq_factor *f, int nrhs_in_F, const double *rhs,
                     int nrhs, int64_t ld_rhs, double *beta, int64_t ld_beta, int max_refine,
                     int mode, double tol, fastlsq_solve_stats *stats)
{
    double *norms = nullptr;
    if (stats) {
        norms = (double *)fl_ws(ctx, FL_WS_NORMS, sizeof(double) * 65);
        if (!norms) return FASTLSQ_ERR_NOMEM;
        cudaMemsetAsync(norms, 0, sizeof(double) * 65, ctx->stream);
    }
    for (int r = 0; r < nrhs; ++r) {
        double *nr = (stats && r == 0) ? norms : nullptr;
        if (f->prec == FASTLSQ_PREC_FP64 && mode != FASTLSQ_REFINE_CGLS)
            FL_TRY(solve_one<double>(ctx, f, nrhs_in_F, r, rhs + r * ld_rhs, beta + r * ld_beta, 0,
                                     mode, tol, nr));
        else if (f->prec == FASTLSQ_PREC_FP64)
            FL_TRY(solve_one<double>(ctx, f, nrhs_in_F, r, rhs + r * ld_rhs, beta + r * ld_beta,
                                     max_refine, mode, tol, nr));
        else
            FL_TRY(solve_one<float>(ctx, f, nrhs_in_F, r, rhs + r * ld_rhs, beta + r * ld_beta,
                                    max_refine, mode, tol, nr));
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        int rc = fastlsq_sync(ctx);
        double h[65] = {0};
        cudaError_t e = cudaMemcpy(h, norms, sizeof(h), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "stats readback");
        for (int i = 0; i < 65; ++i) stats->resid_norm[i] = h[i];
        stats->refine_steps = (f->prec == FASTLSQ_PREC_MIXED || mode == FASTLSQ_REFINE_CGLS) ? max_refine : 0;
        stats->nb = f->nb;
        stats->tensor_core = f->tensor_core;
        stats->status = rc;
        if (rc < 0) return rc;
    }
    return 0;
}

extern "C" int fastlsq_lstsq(fastlsq_ctx *ctx, fastlsq_prec prec, const void *A,
                             fastlsq_dtype a_dtype, int64_t ldA, int64_t n_rows, int64_t n_feat,
                             double mu, const double *rhs, int32_t nrhs, int64_t ld_rhs,
                             double *beta, int64_t ld_beta, const double *A_refine,
                             int64_t ld_refine, int32_t max_refine, int32_t refine_mode,
                             double refine_tol, fastlsq_factor **keep, fastlsq_solve_stats *stats)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    if (keep) *keep = nullptr;
    if (prec != FASTLSQ_PREC_FP64 && prec != FASTLSQ_PREC_MIXED)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: unknown precision");
    if (prec == FASTLSQ_PREC_FP64 && a_dtype != FASTLSQ_F64)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: FP64 precision needs an F64 matrix");
    if (n_rows < 0 || n_feat < 1 || n_feat > FL_MAX_FEAT || ldA < n_rows || nrhs < 0 ||
        (nrhs > 0 && (ld_rhs < n_rows || ld_beta < n_feat)) || mu < 0 || !std::isfinite(mu))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: bad sizes");
    if (refine_mode != FASTLSQ_REFINE_CLASSICAL && refine_mode != FASTLSQ_REFINE_CGLS)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: refine_mode");
    if (max_refine < 0 || max_refine > (refine_mode == FASTLSQ_REFINE_CGLS ? 64 : 7))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: max_refine out of range");
    const int64_t m_aug = n_rows + (mu > 0 ? n_feat : 0);
    if (m_aug < n_feat)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: %lld rows < %lld features needs mu > 0",
                       (long long)n_rows, (long long)n_feat);
    if (!A || (nrhs > 0 && (!rhs || !beta))) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: null array");
    if ((prec == FASTLSQ_PREC_MIXED || refine_mode == FASTLSQ_REFINE_CGLS) && max_refine > 0 &&
        !A_refine && !(prec == FASTLSQ_PREC_FP64))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: refinement needs the FP64 operator");
    if (A_refine && ld_refine < n_rows) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: ld_refine");

    const size_t elem = (prec == FASTLSQ_PREC_FP64) ? 8 : 4;
    const int nb = fl_panel_capacity_nb(ctx, m_aug, elem);
    if (nb == 0)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "lstsq: %lld rows exceed the panel capacity",
                       (long long)m_aug);
    fastlsq_factor *f = new (std::nothrow) fastlsq_factor();
    if (!f) return FASTLSQ_ERR_NOMEM;
    f->ctx = ctx;
    f->stream = ctx->stream;
    f->prec = prec;
    f->m = n_rows;
    f->n = n_feat;
    f->m_aug = m_aug;
    f->ld = fl_round_up(m_aug, 4);
    f->mu = mu;
    f->nb = nb;
    f->A_refine = (prec == FASTLSQ_PREC_MIXED) ? A_refine
                                                : (const double *)(A_refine ? A_refine : A);
    f->ld_refine = (prec == FASTLSQ_PREC_MIXED || A_refine) ? ld_refine : ldA;
    // TF32x3 products carry about 2^-22 relative per product, FP32 FMAs 2^-24: where the
    // factor preconditions CGLS (systems with kappa near 1 / eps32), the FP32 update keeps
    // A R^{-1} well conditioned (measured on Sec. 3.8 instances: cond 2-11 vs 10-170), so
    // the panel-by-panel TF32x3 mode serves classically refined factors only; the blocked
    // mode's three-part bf16 products are FP32-accurate and serve both
    f->tensor_core = 0;
    if (prec == FASTLSQ_PREC_MIXED) {
        if (ctx->use_tensor_core == FL_TC_BLOCKED) f->tensor_core = FL_TC_BLOCKED;
        else if (ctx->use_tensor_core == FL_TC_PANEL && refine_mode == FASTLSQ_REFINE_CLASSICAL)
            f->tensor_core = FL_TC_PANEL;
    }
    int rc = 0;
    const int64_t npanels = fl_cdiv(n_feat, nb);
    f->F = fl_alloc(ctx, elem * f->ld * (n_feat + nrhs), &rc);
    if (f->F) f->tau = fl_alloc(ctx, elem * npanels * nb, &rc);
    if (f->tau) f->T = fl_alloc(ctx, elem * npanels * nb * nb, &rc);
    if (f->T && f->tensor_core == FL_TC_BLOCKED)
        f->Tb = fl_alloc(ctx, sizeof(float) * (size_t)fl_cdiv(n_feat, 128) * 128 * 128, &rc);
    if (!f->T || (f->tensor_core == FL_TC_BLOCKED && !f->Tb)) {
        factor_free(f);
        return rc ? rc : FASTLSQ_ERR_NOMEM;
    }
    if (prec == FASTLSQ_PREC_FP64) {
        rc = fl_copy_in<double, double>(ctx, (const double *)A, ldA, n_rows, n_feat, mu, m_aug, rhs,
                                        ld_rhs, nrhs, (double *)f->F, f->ld);
        if (rc == 0)
            rc = fl_factor<double>(ctx, (double *)f->F, f->ld, m_aug, n_feat, nrhs, nb,
                                   (double *)f->tau, (double *)f->T, 0);
    } else {
        if (a_dtype == FASTLSQ_F32)
            rc = fl_copy_in<float, float>(ctx, (const float *)A, ldA, n_rows, n_feat, mu, m_aug, rhs,
                                          ld_rhs, nrhs, (float *)f->F, f->ld);
        else
            rc = fl_copy_in<double, float>(ctx, (const double *)A, ldA, n_rows, n_feat, mu, m_aug,
                                           rhs, ld_rhs, nrhs, (float *)f->F, f->ld);
        if (rc == 0)
            rc = fl_factor<float>(ctx, (float *)f->F, f->ld, m_aug, n_feat, nrhs, nb,
                                  (float *)f->tau, (float *)f->T, f->tensor_core, (float *)f->Tb, &f->has_tb);
    }
    if (rc == 0 && nrhs > 0)
        rc = solve_all(ctx, f, nrhs, rhs, nrhs, ld_rhs, beta, ld_beta,
                       (prec == FASTLSQ_PREC_MIXED || refine_mode == FASTLSQ_REFINE_CGLS) ? max_refine : 0,
                       refine_mode, refine_tol, stats);
    if (rc == 0 && nrhs == 0 && stats) {            // factor only: report the factor's shape
        memset(stats, 0, sizeof(*stats));
        stats->nb = f->nb;
        stats->tensor_core = f->tensor_core;
        stats->status = rc = fastlsq_sync(ctx);
    }
    if (rc < 0 || !keep) {
        factor_free(f);
        return rc;
    }
    *keep = f;
    return rc;
}

extern "C" int fastlsq_factor_solve(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *rhs,
                                    int32_t nrhs, int64_t ld_rhs, double *beta, int64_t ld_beta,
                                    int32_t max_refine, int32_t refine_mode, double refine_tol,
                                    fastlsq_solve_stats *stats)
{
    if (!ctx || !f) return FASTLSQ_ERR_INVALID;
    if (nrhs < 0 || (nrhs > 0 && (!rhs || !beta || ld_rhs < f->m || ld_beta < f->n)))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "factor_solve: bad arguments");
    if (refine_mode != FASTLSQ_REFINE_CLASSICAL && refine_mode != FASTLSQ_REFINE_CGLS)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "factor_solve: refine_mode");
    if (max_refine < 0 || max_refine > (refine_mode == FASTLSQ_REFINE_CGLS ? 64 : 7))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "factor_solve: max_refine out of range");
    const bool refine = (f->prec == FASTLSQ_PREC_MIXED || refine_mode == FASTLSQ_REFINE_CGLS);
    if (refine && max_refine > 0 && !f->A_refine)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "factor_solve: factor has no FP64 operator");
    return solve_all(ctx, f, 0, rhs, nrhs, ld_rhs, beta, ld_beta, refine ? max_refine : 0,
                     refine_mode, refine_tol, stats);
}

int fl_factor_get_r(fastlsq_ctx *ctx, const fastlsq_factor *f, double *R, int64_t ldr);
int fl_factor_trsv64(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *y, double *x, int transpose);

extern "C" int fastlsq_factor_get_r(fastlsq_ctx *ctx, const fastlsq_factor *f, double *R_out, int64_t ld_r)
{
    if (!ctx || !f || !R_out || ld_r < f->n) return FASTLSQ_ERR_INVALID;
    return fl_factor_get_r(ctx, f, R_out, ld_r);
}

extern "C" int fastlsq_factor_trsv(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *y, double *x,
                                   int32_t transpose)
{
    if (!ctx || !f || !y || !x) return FASTLSQ_ERR_INVALID;
    return fl_factor_trsv64(ctx, f, y, x, transpose ? 1 : 0);
}

extern "C" int fastlsq_factor_destroy(fastlsq_factor *f)
{
    factor_free(f);
    return 0;
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
int fl_matvec64(fastlsq_ctx *ctx, const double *A, int64_t ld, int64_t m, int64_t n,
                const double *v, double *out);

template <typename T>
static int backward_t(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *grad_beta, double *v)
{
    const int64_t n = f->n;
    double *v64 = (double *)fl_ws(ctx, FL_WS_SOLVE64, sizeof(double) * 3 * n + 64);
    if (!v64) return FASTLSQ_ERR_NOMEM;
    FL_TRY(fl_trsv_grid<T>(ctx, (const T *)f->F, f->ld, n, grad_beta, v64, v64 + 2 * n, 1));  // R^{-T} g
    return fl_trsv_grid<T>(ctx, (const T *)f->F, f->ld, n, v64, v, v64 + 2 * n, 0);           // R^{-1} (.)
}

extern "C" int fastlsq_backward(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *grad_beta,
                                double *v, double *grad_rhs, const double *A_op, int64_t ld_op,
                                int32_t max_iter, double tol)
{
    if (!ctx || !f || !grad_beta || !v) return FASTLSQ_ERR_INVALID;
    if (max_iter < 0 || max_iter > 64) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "backward: max_iter 0..64");
    // max_iter > 0: PCG on the normal equations with FP64 operator products, for either
    // factor (the two substitutions alone carry about kappa(R)^2 eps of the factor's type)
    if (max_iter > 0) {
        if (!f->A_refine) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "backward: PCG needs the FP64 operator");
        FL_TRY(wait_refine(ctx));
        FL_TRY(fl_normal_pcg(ctx, f, grad_beta, v, max_iter, tol));
    } else if (f->prec == FASTLSQ_PREC_FP64) {
        FL_TRY(backward_t<double>(ctx, f, grad_beta, v));
    } else {
        FL_TRY(backward_t<float>(ctx, f, grad_beta, v));
    }
    if (grad_rhs) {
        const double *Aop = A_op ? A_op : f->A_refine;
        int64_t ld = A_op ? ld_op : f->ld_refine;
        if (!Aop) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "backward: no FP64 operator for A v");
        if (ld < f->m) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "backward: ld_op");
        if (!A_op) FL_TRY(wait_refine(ctx));
        FL_TRY(fl_matvec64(ctx, Aop, ld, f->m, f->n, v, grad_rhs));
    }
    return 0;
}

extern "C" int fastlsq_source_grad(fastlsq_ctx *ctx, const double *x, int64_t n, const double *theta,
                                   int32_t n_src, const double *w, double *dtheta)
{
    if (!ctx || !x || !theta || !w || !dtheta || n < 0) return FASTLSQ_ERR_INVALID;
    return fl_launch_source_grad(ctx, x, n, theta, n_src, w, dtheta);
}

extern "C" int fastlsq_coef_grad(fastlsq_ctx *ctx, const double *x, int64_t n_rows,
                                 const fastlsq_op *op, const double *W, const double *b,
                                 int64_t n_feat, double scale, const double *r, const double *Av,
                                 const double *v, const double *beta, double *grad)
{
    if (!ctx) return FASTLSQ_ERR_INVALID;
    fl_op_params p;
    FL_TRY(fl_pack_op(ctx, op, &p));
    if (!x || !W || !b || !r || !Av || !v || !beta || !grad || n_rows < 0 || n_feat < 1)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "coef_grad: bad arguments");
    return fl_launch_coef_grad(ctx, x, n_rows, p, W, b, n_feat, scale, r, Av, v, beta, grad);
}

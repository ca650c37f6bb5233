// Krylov refinement of least-squares solutions with a low-precision QR factor as
// preconditioner (mixed-precision iterative refinement in the style of
// LSQR/GMRES-IR, Carson & Higham): the operator products and the residual are
// FP64 against the FP64 operator, the preconditioner applies the factor's R.
//
//  * fl_refine_cgls: CGLS on min ||A~ x - b~|| (A~ = [A; sqrt(mu) I], b~ = [b; 0])
//    right-preconditioned by R (x = R^{-1} y), started from the direct solve.
//    Converges to the FP64 least-squares solution also when the residual is large
//    or kappa(A) eps32 > 1, where classical refinement stagnates.
//  * fl_normal_pcg: preconditioned CG on (A~^T A~) v = c with M = R^T R; this is
//    the adjoint solve v = (A^T A + mu I)^{-1} grad_beta of Sec. 2.5 / Sec. 3.8.
//
// Every kernel reads a device flag and returns at once after convergence, so a
// fixed number of launches can be queued (and captured in a CUDA graph) without
// host round trips.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include <cooperative_groups.h>

#include "common.cuh"
#include "dfloat.cuh"
#include "gridsync.cuh"
#include "qr.cuh"

namespace {

struct KryScalars {
    double gamma, gamma0, qq, alpha, beta;
    double obj;      // CGLS: ||r||^2 (from r.r, less each step's decrease alpha gamma);
                     // PCG: the objective decrease accumulated so far
    int done;
    int iters;
    int accumulate;  // 1: obj accumulates (PCG), 0: obj is what remains (CGLS)
};

// A step that changes the objective by less than this fraction of it, while the
// preconditioned residual no longer falls, is below the resolution of FP64: iterating
// further only lets the recurrence drift (kappa ~ 1e8 systems stall at a
// normal-equations residual far above any relative tolerance)
constexpr double KRY_STALL = 1e-15;

constexpr int KV_ROWS = 256;
constexpr int KV_COLS = 128;

// partial sums of A~ v over column chunks (rows < m)
__global__ void __launch_bounds__(KV_ROWS)
k_kry_mv_partial(const double *__restrict__ A, int64_t ld, int64_t m, int64_t n,
                 const double *__restrict__ v, double *__restrict__ part, const KryScalars *st)
{
    if (st && st->done) return;
    __shared__ double sv[KV_COLS];
    const int64_t j0 = (int64_t)blockIdx.y * KV_COLS;
    const int nc = (int)fl_min64(KV_COLS, n - j0);
    for (int t = threadIdx.x; t < nc; t += blockDim.x) sv[t] = v[j0 + t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * KV_ROWS + threadIdx.x;
    if (i >= m) return;
    double acc = 0.0;
    const double *a = A + i + j0 * ld;
#pragma unroll 8
    for (int c = 0; c < nc; ++c) acc = fma(a[(int64_t)c * ld], sv[c], acc);
    part[(int64_t)blockIdx.y * m + i] = acc;
}

// out = A~ v (rhs == nullptr) or out = rhs~ - A~ v
__global__ void k_kry_mv_finish(const double *__restrict__ part, int nsplit, const double *__restrict__ v,
                                const double *__restrict__ rhs, int64_t m, int64_t m_aug,
                                double sqrt_mu, double *__restrict__ out, const KryScalars *st)
{
    if (st && st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m_aug) return;
    double s;
    if (i < m) {
        s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * m + i];
    } else {
        s = sqrt_mu * v[i - m];
    }
    out[i] = rhs ? ((i < m ? rhs[i] : 0.0) - s) : s;
}

// z_j = sum_i A_ij r_i + sqrt(mu) r_{m+j}: one warp per column (columns are contiguous)
__global__ void __launch_bounds__(256)
k_kry_mvt(const double *__restrict__ A, int64_t ld, int64_t m, int64_t n,
          const double *__restrict__ r, double sqrt_mu, int64_t m_aug, double *__restrict__ z,
          const KryScalars *st)
{
    if (st && st->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t j = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    const double *a = A + j * ld;
    double acc0 = 0.0, acc1 = 0.0;
    int64_t i = lane;
    for (; i + 32 < m; i += 64) {
        acc0 = fma(a[i], r[i], acc0);
        acc1 = fma(a[i + 32], r[i + 32], acc1);
    }
    for (; i < m; i += 32) acc0 = fma(a[i], r[i], acc0);
    double acc = acc0 + acc1;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[j] = acc + ((m_aug > m) ? sqrt_mu * r[m + j] : 0.0);
}

constexpr int DOT_THREADS = 256;
constexpr int DOT_BLOCKS = 128;

__global__ void __launch_bounds__(DOT_THREADS)
k_kry_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                  double *__restrict__ part, const KryScalars *st)
{
    if (st && st->done) return;
    __shared__ double red[DOT_THREADS];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * DOT_THREADS + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * DOT_THREADS)
        acc = fma(a[i], b[i], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = DOT_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

enum { OP_INIT = 0, OP_ALPHA = 1, OP_BETA = 2, OP_NORM = 3, OP_OBJ = 4, OP_INIT_ACC = 5 };

// sums the dot partials in a fixed order and advances the scalar recurrence
__global__ void k_kry_scalar(const double *__restrict__ part, int nblk, KryScalars *st, int op,
                             double tol, double *norm_out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (op != OP_INIT && op != OP_INIT_ACC && op != OP_OBJ && st->done) return;
    double d = 0.0;
    for (int b = 0; b < nblk; ++b) d += part[b];
    if (op == OP_INIT || op == OP_INIT_ACC) {
        st->gamma = d;
        st->gamma0 = d;
        st->iters = 0;
        st->done = !(d > 0.0) || !isfinite(d);
        st->accumulate = (op == OP_INIT_ACC);
        st->obj = 0.0;
    } else if (op == OP_OBJ) {
        st->obj = d;
    } else if (op == OP_ALPHA) {
        st->qq = d;
        if (!(d > 0.0) || !isfinite(d)) {
            st->alpha = 0.0;
            st->done = 1;
        } else {
            st->alpha = st->gamma / d;
        }
    } else if (op == OP_BETA) {
        // this step lowered the objective by alpha gamma (CGLS: ||r||^2; PCG: twice the
        // quadratic form's decrease)
        const double dec = st->alpha * st->gamma;
        st->obj = st->accumulate ? st->obj + dec : st->obj - dec;
        // stalled: the objective no longer moves AND the preconditioned residual has
        // stopped falling (a flat objective alone can hide progress along directions
        // that barely change it)
        const bool stalled = !(dec > KRY_STALL * st->obj) && d > 0.5 * st->gamma;
        st->beta = d / st->gamma;
        st->gamma = d;
        st->iters += 1;
        if (!(d > tol * tol * st->gamma0) || !isfinite(d)) st->done = 1;
        if (stalled) st->done = 1;                        // (an estimate <= 0 never fires)
    } else if (op == OP_NORM) {
        if (norm_out) *norm_out = sqrt(d);
    }
}

// y += sign * alpha * x
__global__ void k_kry_axpy(double *__restrict__ y, const double *__restrict__ x, int64_t n,
                           const KryScalars *st, double sign)
{
    if (st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = fma(sign * st->alpha, x[i], y[i]);
}

// p = s + beta * p
__global__ void k_kry_xpby(double *__restrict__ p, const double *__restrict__ s, int64_t n,
                           const KryScalars *st)
{
    if (st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = fma(st->beta, p[i], s[i]);
}

__global__ void k_kry_copy_sub(double *__restrict__ dst, const double *__restrict__ a,
                               const double *__restrict__ b, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = b ? a[i] - b[i] : a[i];
}

// ---------------------------------------------------------------------------
// FP64 triangular solves with the factor's R (entries of type T promoted to
// double): R x = y (transpose 0) or R^T x = y.  Applying R^{-1} in FP64 keeps the
// preconditioner a fixed linear operator even when kappa(R) eps32 >> 1, and the
// FP64 path gets LAPACK-grade backward stability: every 64 x 64 diagonal block is
// solved by substitution (no explicit inverse, whose error grows with the block's
// condition number), the off-diagonal blocks are applied as FP64 mat-vecs.
//
//  * k_trsv_cluster: one cluster of up to 16 CTAs.  64-row block b belongs to
//    rank b % CS, which keeps its diagonal block and its rows of the running
//    right-hand side w in shared memory.  Per block: the owner's warp 0 solves the
//    diagonal block and writes x_b into every rank's shared copy of x (DSMEM);
//    one cluster barrier; every rank removes x_b's contribution from its own
//    remaining rows.  No grid barrier and no global scratch.
//  * k_trsv_grid: the same blocked substitution on a cooperative grid for R too
//    large for the cluster's shared memory (two grid barriers per block; each
//    barrier spins for at most about a second, then raises the device flag and
//    the kernel returns).
// ---------------------------------------------------------------------------
constexpr int TG_BS = 64;
constexpr int TG_THREADS = 256;
constexpr int TC_THREADS = 512;
constexpr int TS_LD = TG_BS + 1;        // padded column stride of a staged diagonal block
constexpr int TC_MAX_CS = 16;

// Stage diagonal block b as the "effective" triangle E in column-major layout
// E[j * TS_LD + i]: E = D (upper) or D^T (lower, transpose).  Ragged rows/cols
// beyond n become the identity so that the padded unknowns solve to zero.
template <typename T, typename A>
__device__ __forceinline__ void trsv_stage_diag(const T *__restrict__ F, int64_t ld, int64_t n, int64_t r0,
                                                int transpose, A *E, int tid, int nthreads)
{
    const int nb = (int)fl_min64(TG_BS, n - r0);
    for (int idx = tid; idx < TG_BS * TG_BS; idx += nthreads) {
        // consecutive threads read consecutive addresses of F in both cases
        const int a = idx % TG_BS, c = idx / TG_BS;          // F row r0 + a, F column r0 + c
        A v;
        if (a < nb && c < nb) v = (a <= c) ? (A)F[(r0 + a) + (r0 + c) * ld] : A(0);   // R is D's upper triangle
        else v = (a == c) ? A(1) : A(0);
        if (!transpose) E[c * TS_LD + a] = v;                // E(i=a, j=c) = D(a, c)
        else E[a * TS_LD + c] = v;                           // E(i=c, j=a) = D(a, c)
    }
}

// Substitution on one staged 64 x 64 triangle by one warp.  Lane l holds rows l
// and l + 32 of the running right-hand side (w0, w1) and returns x in (w0, w1).
// Upper: j = 63..0, x_j = w_j / E_jj, w_i -= E_ij x_j (i < j).  Lower: j = 0..63,
// i > j.  x_j is formed as w_j * (1 / E_jj) (at most two roundings) so that the
// dependent chain per unknown is one multiply, one shuffle and one FMA.
template <typename A>
__device__ __forceinline__ void trsv_diag_warp(const A *E, int lower, int lane, A &w0, A &w1)
{
    const A rinv0 = A(1) / E[lane * TS_LD + lane];
    const A rinv1 = A(1) / E[(lane + 32) * TS_LD + lane + 32];
    A x0 = A(0), x1 = A(0);
    if (!lower) {
#pragma unroll
        for (int j = TG_BS - 1; j >= 0; --j) {
            const A t = (j < 32) ? w0 * rinv0 : w1 * rinv1;
            const A xj = __shfl_sync(0xffffffffu, t, j & 31);
            if (lane == (j & 31)) { if (j < 32) x0 = xj; else x1 = xj; }
            const A *col = E + j * TS_LD;
            if (lane < j) w0 = fma(-col[lane], xj, w0);
            if (lane + 32 < j) w1 = fma(-col[lane + 32], xj, w1);
        }
    } else {
#pragma unroll
        for (int j = 0; j < TG_BS; ++j) {
            const A t = (j < 32) ? w0 * rinv0 : w1 * rinv1;
            const A xj = __shfl_sync(0xffffffffu, t, j & 31);
            if (lane == (j & 31)) { if (j < 32) x0 = xj; else x1 = xj; }
            const A *col = E + j * TS_LD;
            if (lane > j) w0 = fma(-col[lane], xj, w0);
            if (lane + 32 > j) w1 = fma(-col[lane + 32], xj, w1);
        }
    }
    w0 = x0;
    w1 = x1;
}

struct TrsvClusterSmem {
    // [nown][TG_BS * TS_LD] staged diagonal blocks, [nown][TG_BS] w, [nblk * TG_BS] x
    static __host__ __device__ size_t bytes(int nown, int64_t nblk, size_t elem)
    {
        return elem * ((size_t)nown * (TG_BS * TS_LD + TG_BS) + (size_t)nblk * TG_BS);
    }
};

template <typename T, typename A>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_trsv_cluster(const T *__restrict__ F, int64_t ld, int64_t n, const double *__restrict__ y,
               double *__restrict__ x, int transpose, int *flag, const KryScalars *st)
{
    if (st && st->done) return;              // same value in every CTA of the cluster
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char tsm_raw[];
    A *tsm = reinterpret_cast<A *>(tsm_raw);
    __shared__ A red[2][4 * TG_BS];
    const int rank = (int)cluster.block_rank();
    const int CS = (int)cluster.num_blocks();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t nblk = (n + TG_BS - 1) / TG_BS;
    const int nown = (int)((nblk - rank + CS - 1) / CS);
    const int nown_max = (int)((nblk + CS - 1) / CS);
    A *Es = tsm;
    A *ws = Es + (size_t)nown_max * TG_BS * TS_LD;
    A *xs = ws + (size_t)nown_max * TG_BS;
    for (int lb = 0; lb < nown; ++lb) {
        const int64_t r0 = (int64_t)(rank + lb * CS) * TG_BS;
        trsv_stage_diag(F, ld, n, r0, transpose, Es + (size_t)lb * TG_BS * TS_LD, tid, TC_THREADS);
        for (int i = tid; i < TG_BS; i += TC_THREADS) ws[lb * TG_BS + i] = (r0 + i < n) ? (A)y[r0 + i] : A(0);
    }
    cluster.sync();                          // every rank resident before the first DSMEM store
    for (int64_t s = 0; s < nblk; ++s) {
        const int64_t b = transpose ? s : nblk - 1 - s;
        const int64_t r0 = b * TG_BS;
        const int nb = (int)fl_min64(TG_BS, n - r0);
        if ((int)(b % CS) == rank && warp == 0) {
            const int lb = (int)(b / CS);
            A w0 = ws[lb * TG_BS + lane], w1 = ws[lb * TG_BS + lane + 32];
            trsv_diag_warp(Es + (size_t)lb * TG_BS * TS_LD, transpose, lane, w0, w1);
            if (!isfinite(w0) || !isfinite(w1)) atomicCAS(flag, 0, FL_DEVERR_NONFINITE);
            for (int rr = 0; rr < CS; ++rr) {
                A *dst = cluster.map_shared_rank(xs, rr);
                dst[r0 + lane] = w0;
                dst[r0 + lane + 32] = w1;
            }
        }
        cluster.sync();
        const A *xb = xs + r0;
        if (!transpose) {
            // owned rows of blocks b' < b: w_i -= sum_c R(i, r0 + c) x_c; two column halves
            const int row = tid & (4 * TG_BS - 1), half = tid / (4 * TG_BS);
            const int lb = row / TG_BS, ri = row % TG_BS;
            const int64_t bb = (int64_t)rank + (int64_t)lb * CS;
            A acc = A(0);
            if (lb < nown && bb < b) {
                const T *a = F + (bb * TG_BS + ri) + (r0 + half * 32) * ld;
                const int c1 = fl_min64(32, nb - half * 32);
                T v[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = (c < c1) ? a[(int64_t)c * ld] : (T)0;
#pragma unroll
                for (int c = 0; c < 32; ++c) acc = fma((A)v[c], xb[half * 32 + c], acc);
            }
            red[half][row] = acc;
            __syncthreads();
            if (tid < 4 * TG_BS && lb < nown && bb < b) ws[row] -= red[0][row] + red[1][row];
        } else {
            // owned rows i of blocks b' > b: w_i -= sum_c R(r0 + c, i) x_c; warp per 16 rows,
            // lanes over c (contiguous in column i of F)
            const int nrow_own = nown * TG_BS;
            for (int base = warp * 16; base < nrow_own; base += (TC_THREADS / 32) * 16) {
                A acc[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int row = base + q;
                    const int lb = row / TG_BS, ri = row % TG_BS;
                    const int64_t bb = (int64_t)rank + (int64_t)lb * CS;
                    const int64_t i = bb * TG_BS + ri;
                    acc[q] = A(0);
                    if (row < nrow_own && bb > b && i < n) {
                        const T *a = F + r0 + i * ld;
                        const A v0 = (lane < nb) ? (A)a[lane] : A(0);
                        const A v1 = (lane + 32 < nb) ? (A)a[lane + 32] : A(0);
                        acc[q] = fma(v0, xb[lane], v1 * xb[lane + 32]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
                if (lane < 16) {
                    A mine = acc[0];
#pragma unroll
                    for (int q = 1; q < 16; ++q) if (lane == q) mine = acc[q];
                    const int row = base + lane;
                    const int lb = row / TG_BS;
                    const int64_t bb = (int64_t)rank + (int64_t)lb * CS;
                    if (row < nrow_own && bb > b) ws[row] -= mine;
                }
            }
        }
        __syncthreads();
    }
    for (int lb = 0; lb < nown; ++lb) {
        const int64_t r0 = (int64_t)(rank + lb * CS) * TG_BS;
        for (int i = tid; i < TG_BS; i += TC_THREADS)
            if (r0 + i < n) x[r0 + i] = (double)xs[r0 + i];
    }
}

template <typename T>
__global__ void __launch_bounds__(TG_THREADS, 1)
k_trsv_grid(const T *__restrict__ F, int64_t ld, int64_t n, const double *__restrict__ y,
            double *__restrict__ x, double *__restrict__ work, int transpose, GridBar *bar, int *flag,
            const KryScalars *st)
{
    if (st && st->done) return;              // same value in every CTA
    __shared__ double E[TG_BS * TS_LD];
    __shared__ volatile int s_abort;
    const unsigned G = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_abort = 0;
    for (int64_t i = (int64_t)blockIdx.x * TG_THREADS + threadIdx.x; i < n; i += (int64_t)G * TG_THREADS)
        work[i] = y[i];
    if (!grid_sync(bar, G, flag, &s_abort)) return;
    const int64_t nblk = (n + TG_BS - 1) / TG_BS;
    for (int64_t step = 0; step < nblk; ++step) {
        const int64_t b = transpose ? step : nblk - 1 - step;
        const int64_t r0 = b * TG_BS, r1 = fl_min64(n, r0 + TG_BS);
        const int nb = (int)(r1 - r0);
        if (blockIdx.x == 0) {
            trsv_stage_diag(F, ld, n, r0, transpose, E, threadIdx.x, TG_THREADS);
            __syncthreads();
            if (warp == 0) {
                double w0 = (lane < nb) ? work[r0 + lane] : 0.0;
                double w1 = (lane + 32 < nb) ? work[r0 + lane + 32] : 0.0;
                trsv_diag_warp(E, transpose, lane, w0, w1);
                if (!isfinite(w0) || !isfinite(w1)) atomicCAS(flag, 0, FL_DEVERR_NONFINITE);
                if (lane < nb) x[r0 + lane] = w0;
                if (lane + 32 < nb) x[r0 + lane + 32] = w1;
            }
        }
        if (!grid_sync(bar, G, flag, &s_abort)) return;
        if (!transpose) {
            // rows i < r0: work_i -= sum_c R(i, r0 + c) x_{r0 + c}   (thread per row, coalesced)
            for (int64_t i = (int64_t)blockIdx.x * TG_THREADS + threadIdx.x; i < r0;
                 i += (int64_t)G * TG_THREADS) {
                double acc = 0.0;
#pragma unroll 16
                for (int c = 0; c < nb; ++c) acc = fma((double)F[i + (r0 + c) * ld], x[r0 + c], acc);
                work[i] -= acc;
            }
        } else {
            // rows i >= r1: work_i -= sum_c R(r0 + c, i) x_{r0 + c}   (warp per row, coalesced)
            for (int64_t i = r1 + (int64_t)blockIdx.x * (TG_THREADS / 32) + warp; i < n;
                 i += (int64_t)G * (TG_THREADS / 32)) {
                double acc = 0.0;
                for (int c = lane; c < nb; c += 32) acc = fma((double)F[(r0 + c) + i * ld], x[r0 + c], acc);
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) work[i] -= acc;
            }
        }
        if (!grid_sync(bar, G, flag, &s_abort)) return;
    }
}

struct KryBufs {
    double *r, *s, *p, *t, *q, *z, *part;
    KryScalars *st;
    void *tf;   // factor-type temporary [n]
    double *work;
    GridBar *bar;
};

int kry_bufs(fastlsq_ctx *ctx, const fastlsq_factor *f, KryBufs *B)
{
    const int64_t n = f->n, m_aug = f->m_aug;
    const int nsplit = (int)fl_cdiv(n, KV_COLS);
    size_t nd = (size_t)(2 * m_aug + 5 * n) + (size_t)nsplit * f->m + DOT_BLOCKS + 64;
    double *base = (double *)fl_ws(ctx, FL_WS_KRYLOV, sizeof(double) * nd + sizeof(KryScalars) + 64);
    void *tf = fl_ws(ctx, FL_WS_VEC1, 8 * (size_t)n + 64);
    if (!base || !tf) return FASTLSQ_ERR_NOMEM;
    B->r = base;
    B->q = B->r + m_aug;
    B->s = B->q + m_aug;
    B->p = B->s + n;
    B->t = B->p + n;
    B->z = B->t + n;
    B->part = B->z + n;
    B->work = B->part + (size_t)nsplit * f->m + DOT_BLOCKS + 8;
    B->st = (KryScalars *)(B->work + n + 8);
    B->tf = tf;
    B->bar = (GridBar *)ctx->d_grid_bar;
    return 0;
}

int kry_mv(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *v, const double *rhs,
           double *out, const KryBufs &B, const KryScalars *st)
{
    const int nsplit = (int)fl_cdiv(f->n, KV_COLS);
    FL_PROF_N(ctx, FASTLSQ_K_KRYLOV, 2);
    k_kry_mv_partial<<<dim3((unsigned)fl_cdiv(f->m, KV_ROWS), (unsigned)nsplit), KV_ROWS, 0, ctx->stream>>>(
        f->A_refine, f->ld_refine, f->m, f->n, v, B.part, st);
    k_kry_mv_finish<<<(unsigned)fl_cdiv(f->m_aug, 256), 256, 0, ctx->stream>>>(
        B.part, nsplit, v, rhs, f->m, f->m_aug, f->mu > 0 ? sqrt(f->mu) : 0.0, out, st);
    FL_CHECK_LAUNCH(ctx, "krylov mv");
    return 0;
}

int kry_mvt(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *r, double *z, const KryScalars *st)
{
    FL_PROF(ctx, FASTLSQ_K_KRYLOV);
    k_kry_mvt<<<(unsigned)fl_cdiv(f->n, 8), 256, 0, ctx->stream>>>(
        f->A_refine, f->ld_refine, f->m, f->n, r, f->mu > 0 ? sqrt(f->mu) : 0.0, f->m_aug, z, st);
    FL_CHECK_LAUNCH(ctx, "krylov mvt");
    return 0;
}

int kry_dot(fastlsq_ctx *ctx, const double *a, const double *b, int64_t n, const KryBufs &B, int op,
            double tol, double *norm_out, const KryScalars *skip)
{
    FL_PROF_N(ctx, FASTLSQ_K_KRYLOV, 2);
    k_kry_dot_partial<<<DOT_BLOCKS, DOT_THREADS, 0, ctx->stream>>>(a, b, n, B.part, skip);
    k_kry_scalar<<<1, 32, 0, ctx->stream>>>(B.part, DOT_BLOCKS, B.st, op, tol, norm_out);
    FL_CHECK_LAUNCH(ctx, "krylov dot");
    return 0;
}

}  // namespace

// x = R^{-1} y (transpose 0) or R^{-T} y in FP64 with the factor's R (type T);
// work: [n] FP64 scratch (grid variant only); skip: optional device flag that
// makes the call a no-op.
template <typename T>
int fl_trsv_grid(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t n, const double *y, double *x,
                 double *work, int transpose, const void *skip_scalars, int arith)
{
    FL_PROF(ctx, FASTLSQ_K_TRSV);
    int *flag = ctx->d_flag;
    const KryScalars *st = (const KryScalars *)skip_scalars;
    const int64_t nblk = fl_cdiv(n, TG_BS);
    const int CS = (int)std::min<int64_t>(TC_MAX_CS, nblk);
    const int nown_max = (int)fl_cdiv(nblk, CS);
    // FP32 or double-float arithmetic only on request and only for an FP32 factor
    const int mode = std::is_same<T, float>::value ? ((arith == FL_ARITH_F32 || arith == FL_ARITH_DF) ? arith : 0) : 0;
    const size_t elem = (mode == FL_ARITH_F32) ? sizeof(float) : sizeof(double);
    const size_t smem = TrsvClusterSmem::bytes(nown_max, nblk, elem);
    using K = void (*)(const T *, int64_t, int64_t, const double *, double *, int, int *, const KryScalars *);
    K kern = (mode == FL_ARITH_F32) ? (K)k_trsv_cluster<T, float>
             : (mode == FL_ARITH_DF) ? (K)k_trsv_cluster<T, dfl> : (K)k_trsv_cluster<T, double>;
    static FlOncePerDevice attr_once[3];
    if (nown_max <= 4 && smem + elem * 2 * 4 * TG_BS <= (size_t)ctx->max_smem_optin) {
        if (attr_once[mode].pending(ctx->device)) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 ctx->max_smem_optin - (int)(elem * 2 * 4 * TG_BS));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return fl_cuda(ctx, e, "cudaFuncSetAttribute");
            attr_once[mode].done(ctx->device);
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CS);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = ctx->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = CS;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, F, ld, n, y, x, transpose, flag, st);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "cluster triangular solve");
        return 0;
    }
    GridBar *bar = (GridBar *)ctx->d_grid_bar;
    void *args[] = {(void *)&F, (void *)&ld, (void *)&n, (void *)&y, (void *)&x, (void *)&work,
                    (void *)&transpose, (void *)&bar, (void *)&flag, (void *)&st};
    // a few dozen CTAs: the per-block updates are small and barrier cost grows with the grid
    const unsigned G = (unsigned)std::min<int64_t>(ctx->num_sms, std::max<int64_t>(8, nblk));
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_trsv_grid<T>, dim3(G),
                                                dim3(TG_THREADS), args, 0, ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "grid triangular solve");
    return 0;
}
template int fl_trsv_grid<float>(fastlsq_ctx *, const float *, int64_t, int64_t, const double *,
                                 double *, double *, int, const void *, int);
template int fl_trsv_grid<double>(fastlsq_ctx *, const double *, int64_t, int64_t, const double *,
                                  double *, double *, int, const void *, int);

namespace {

// out = R^{-1} in (transpose = 0) or R^{-T} in with the factor's R: in FP64, or, as the
// preconditioner of CGLS and PCG with an FP32 factor (precond), in double-float
// arithmetic when the context allows it (about 48 bits: the preconditioner need only
// stay the same linear map to well below the FP32 factor's own error, and the FP64
// residuals and products of the Krylov method set the accuracy of the result)
template <typename T>
int kry_prec(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *in, double *out, int transpose,
             const KryBufs &B, bool precond = true)
{
    const int arith = (precond && ctx->krylov_df && std::is_same<T, float>::value) ? FL_ARITH_DF : 0;
    return fl_trsv_grid<T>(ctx, (const T *)f->F, f->ld, f->n, in, out, B.work, transpose, B.st, arith);
}

template <typename T>
int refine_cgls_t(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *rhs64, double *x,
                  int max_iter, double tol, double *norms)
{
    KryBufs B;
    FL_TRY(kry_bufs(ctx, f, &B));
    const int64_t n = f->n, m_aug = f->m_aug;
    const unsigned gn = (unsigned)fl_cdiv(n, 256), gm = (unsigned)fl_cdiv(m_aug, 256);
    cudaMemsetAsync(B.st, 0, sizeof(KryScalars), ctx->stream);
    // r = b~ - A~ x ; s = R^{-T} A~^T r ; p = s ; gamma = s.s
    FL_TRY(kry_mv(ctx, f, x, rhs64, B.r, B, nullptr));
    if (norms) FL_TRY(kry_dot(ctx, B.r, B.r, m_aug, B, OP_NORM, 0.0, norms, nullptr));
    FL_TRY(kry_mvt(ctx, f, B.r, B.z, nullptr));
    FL_TRY(kry_prec<T>(ctx, f, B.z, B.s, 1, B));
    k_kry_copy_sub<<<gn, 256, 0, ctx->stream>>>(B.p, B.s, nullptr, n);
    ctx->prof.launches[FASTLSQ_K_KRYLOV] += 1;
    FL_TRY(kry_dot(ctx, B.s, B.s, n, B, OP_INIT, tol, nullptr, nullptr));
    FL_TRY(kry_dot(ctx, B.r, B.r, m_aug, B, OP_OBJ, tol, nullptr, nullptr));
    for (int it = 0; it < max_iter; ++it) {
        FL_TRY(kry_prec<T>(ctx, f, B.p, B.t, 0, B));                 // t = R^{-1} p
        FL_TRY(kry_mv(ctx, f, B.t, nullptr, B.q, B, B.st));           // q = A~ t
        FL_TRY(kry_dot(ctx, B.q, B.q, m_aug, B, OP_ALPHA, tol, nullptr, B.st));
        k_kry_axpy<<<gn, 256, 0, ctx->stream>>>(x, B.t, n, B.st, 1.0);
        k_kry_axpy<<<gm, 256, 0, ctx->stream>>>(B.r, B.q, m_aug, B.st, -1.0);
        FL_TRY(kry_mvt(ctx, f, B.r, B.z, B.st));                      // z = A~^T r
        FL_TRY(kry_prec<T>(ctx, f, B.z, B.s, 1, B));                  // s = R^{-T} z
        FL_TRY(kry_dot(ctx, B.s, B.s, n, B, OP_BETA, tol, nullptr, B.st));
        k_kry_xpby<<<gn, 256, 0, ctx->stream>>>(B.p, B.s, n, B.st);
        ctx->prof.launches[FASTLSQ_K_KRYLOV] += 3;
        if (norms && it + 1 < 64) FL_TRY(kry_dot(ctx, B.r, B.r, m_aug, B, OP_NORM, 0.0, norms + it + 1, B.st));
        FL_CHECK_LAUNCH(ctx, "cgls");
    }
    return 0;
}

template <typename T>
int normal_pcg_t(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *c, double *v, int max_iter,
                 double tol)
{
    KryBufs B;
    FL_TRY(kry_bufs(ctx, f, &B));
    const int64_t n = f->n;
    const unsigned gn = (unsigned)fl_cdiv(n, 256);
    cudaMemsetAsync(B.st, 0, sizeof(KryScalars), ctx->stream);
    // v0 = M^{-1} c ; z = c - A~^T A~ v0 ; y(=s) = M^{-1} z ; p = y ; rho = z.y
    FL_TRY(kry_prec<T>(ctx, f, c, B.t, 1, B));
    FL_TRY(kry_prec<T>(ctx, f, B.t, v, 0, B));
    FL_TRY(kry_mv(ctx, f, v, nullptr, B.q, B, nullptr));
    FL_TRY(kry_mvt(ctx, f, B.q, B.r, nullptr));                       // r (n-space) = A~^T A~ v0
    k_kry_copy_sub<<<gn, 256, 0, ctx->stream>>>(B.z, c, B.r, n);      // z = c - A~^T A~ v0
    FL_TRY(kry_prec<T>(ctx, f, B.z, B.t, 1, B));
    FL_TRY(kry_prec<T>(ctx, f, B.t, B.s, 0, B));
    k_kry_copy_sub<<<gn, 256, 0, ctx->stream>>>(B.p, B.s, nullptr, n);
    ctx->prof.launches[FASTLSQ_K_KRYLOV] += 2;
    FL_TRY(kry_dot(ctx, B.z, B.s, n, B, OP_INIT_ACC, tol, nullptr, nullptr));
    for (int it = 0; it < max_iter; ++it) {
        FL_TRY(kry_mv(ctx, f, B.p, nullptr, B.q, B, B.st));
        FL_TRY(kry_mvt(ctx, f, B.q, B.r, B.st));                      // w = A~^T A~ p (in r)
        FL_TRY(kry_dot(ctx, B.p, B.r, n, B, OP_ALPHA, tol, nullptr, B.st));
        k_kry_axpy<<<gn, 256, 0, ctx->stream>>>(v, B.p, n, B.st, 1.0);
        k_kry_axpy<<<gn, 256, 0, ctx->stream>>>(B.z, B.r, n, B.st, -1.0);
        FL_TRY(kry_prec<T>(ctx, f, B.z, B.t, 1, B));
        FL_TRY(kry_prec<T>(ctx, f, B.t, B.s, 0, B));
        FL_TRY(kry_dot(ctx, B.z, B.s, n, B, OP_BETA, tol, nullptr, B.st));
        k_kry_xpby<<<gn, 256, 0, ctx->stream>>>(B.p, B.s, n, B.st);
        ctx->prof.launches[FASTLSQ_K_KRYLOV] += 3;
        FL_CHECK_LAUNCH(ctx, "normal pcg");
    }
    return 0;
}

}  // namespace

int fl_refine_cgls(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *rhs64, double *beta64,
                   int max_iter, double tol, double *norms_dev)
{
    if (!f->A_refine) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "CGLS refinement needs the FP64 operator");
    if (f->prec == FASTLSQ_PREC_FP64)
        return refine_cgls_t<double>(ctx, f, rhs64, beta64, max_iter, tol, norms_dev);
    return refine_cgls_t<float>(ctx, f, rhs64, beta64, max_iter, tol, norms_dev);
}

int fl_normal_pcg(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *c64, double *v64,
                  int max_iter, double tol)
{
    if (!f->A_refine) return fl_fail(ctx, FASTLSQ_ERR_INVALID, "PCG adjoint needs the FP64 operator");
    if (f->prec == FASTLSQ_PREC_FP64) return normal_pcg_t<double>(ctx, f, c64, v64, max_iter, tol);
    return normal_pcg_t<float>(ctx, f, c64, v64, max_iter, tol);
}

namespace {
template <typename T>
__global__ void k_get_r(const T *__restrict__ F, int64_t ld, int64_t n, double *__restrict__ R, int64_t ldr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j = blockIdx.y;
    if (i >= n || j >= n) return;
    R[i + j * ldr] = (i <= j) ? (double)F[i + j * ld] : 0.0;
}
}  // namespace

int fl_factor_get_r(fastlsq_ctx *ctx, const fastlsq_factor *f, double *R, int64_t ldr)
{
    FL_PROF(ctx, FASTLSQ_K_VECTOR);
    dim3 grid((unsigned)fl_cdiv(f->n, 256), (unsigned)f->n);
    if (f->prec == FASTLSQ_PREC_FP64)
        k_get_r<double><<<grid, 256, 0, ctx->stream>>>((const double *)f->F, f->ld, f->n, R, ldr);
    else
        k_get_r<float><<<grid, 256, 0, ctx->stream>>>((const float *)f->F, f->ld, f->n, R, ldr);
    FL_CHECK_LAUNCH(ctx, "get_r");
    return 0;
}

int fl_factor_trsv64(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *y, double *x, int transpose)
{
    KryBufs B;
    FL_TRY(kry_bufs(ctx, f, &B));
    cudaMemsetAsync(B.st, 0, sizeof(KryScalars), ctx->stream);
    if (f->prec == FASTLSQ_PREC_FP64) return kry_prec<double>(ctx, f, y, x, transpose, B, false);
    return kry_prec<float>(ctx, f, y, x, transpose, B, false);
}

// Batched inverse problem with pre-factored operators (Sec. 3.8 in steady form;
// Sec. 2.5: gradients through the pre-factored solve, two triangular solves per
// evaluation): many instances of uneven size, every gradient evaluation of the whole
// batch in ONE persistent launch.
//
// fastlsq_inverse_prepare factors each instance once (FP64 Householder QR of
// [A; sqrt(mu) I], kept: the checkpoint the evaluations reuse; several instances at a
// time on worker streams), by default forms Qi = the interior rows of Q [I; 0] from the
// kept factor (thin-Q plan, evaluated by k_inv_eval_q below), and tabulates the sensor
// matrix H_s (n_sens x n_feat, FP64).  With the reflector plan,
// fastlsq_inverse_eval launches k_inv_eval: a grid of persistent clusters of C CTAs
// (C = 1, 2 or 4) that take instances from a device-side queue (one atomic counter,
// instances in decreasing order of m_aug n, so the longest start first); a cluster runs
// an instance's whole evaluation with its vectors in shared memory, the m_aug-vectors
// dealt over the ranks in stripes of 32 rows:
//   y   = [s(x_int; theta); 0 (u = 0 rows); 0 (sqrt(mu) rows)]
//   y  <- Q^T y                       (the factor's reflectors, panel by panel; per
//                                      panel the ranks' partial V^T y exchanged
//                                      through distributed shared memory)
//   beta = R^{-1} y[0:n]              (blocked substitution, rank 0)
//   u_s = H_s beta, L = mean (u_s - y_obs)^2, g = dL/du_s
//   w   = R^{-T} (H_s^T g)            (rank 0)
//   z   = Q [w; 0]                    (= A (A^T A + mu I)^{-1} H_s^T g = dL/d rhs)
//   dL/dtheta = sum_{i < n_int} z_i ds(x_i; theta)/dtheta   (ranks' sums in rank order)
// Clusters do not wait on one another: the queue is their only shared state; inside a
// cluster the ranks meet at hardware cluster barriers, which the ranks, launched
// together, always reach.  The launch allocates nothing and synchronises nothing on the
// host, so a caller can capture it in a CUDA graph and replay it with new theta and
// y_obs.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "qr.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int IB_MAX_SRC = 8;
constexpr int IB_MAX_SENS = 256;
constexpr int IB_NB = 32;              // largest panel width of an FP64 factor
constexpr int IB_SETUP_WORKERS = 4;    // concurrent factorisations in the setup

struct InvDesc {
    int64_t n_int, n_feat, n_sens, m_aug, ld;
    int nb;
    double scale;
    const double *x_int, *theta, *y_obs, *H;      // H: [n_sens][n_feat]
    const double *F, *T;                          // factor (V below, R above), T blocks
    const double *Q;                              // thin-Q form: rows [0, n_int) of Q [I; 0]
    int64_t ldq;
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

// Rows of an instance's m_aug-vectors held by one CTA of a cluster of C: stripes of 32
// rows dealt round-robin (stripe t of rank r is rows 32 (t C + r) .. + 31), kept at local
// index 32 t + (row & 31).  Every panel's rows [k, m_aug) are then shared almost evenly
// by the cluster, and a warp's 32 consecutive local rows are 32 consecutive rows of the
// factor (coalesced).  C = 1 is the identity.
template <int C>
struct IbRows {
    int rank;
    __device__ __forceinline__ int64_t glob(int64_t lr) const
    {
        return (C == 1) ? lr : (((lr >> 5) * C + rank) << 5) + (lr & 31);
    }
    // first local index whose row is >= k
    __device__ __forceinline__ int64_t first(int64_t k) const
    {
        if (C == 1) return k;
        const int64_t sk = k >> 5;
        const int64_t t = (sk >= rank) ? (sk - rank + C - 1) / C : 0;
        return (t * C + rank == sk) ? (t << 5) + (k & 31) : (t << 5);
    }
};

// The cluster's shared state of one CTA: the exchange buffers written by the other
// ranks through distributed shared memory.
struct IbXchg {
    double *xs;        // [2][C][32]  per-panel partial sums s = V^T y, double-buffered
    double *xd;        // [C][4 IB_MAX_SRC]  per-rank partial gradients
    int flip;          // which half of xs the next exchange uses
};

// y <- Q^T y (transpose) or Q y on the cluster's distributed vector y (this CTA's rows,
// local indices), FP64.  Per panel: s = V^T y (each thread its rows, warp
// reduce-scatter, warps summed in order; with C > 1 the ranks' sums exchanged and
// added in rank order, so every rank holds the same s), w = T^T s or T s, y -= V w.
template <int THREADS, int C>
__device__ void ib_apply_q(const InvDesc &D, const IbRows<C> &rows, double *y, double *red, double *wv,
                           IbXchg &xc, bool transpose)
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
        const int64_t lr0 = rows.first(k);
        double acc[IB_NB];
#pragma unroll
        for (int l = 0; l < IB_NB; ++l) acc[l] = 0.0;
        for (int64_t lr = lr0 + tid;; lr += THREADS) {
            const int64_t i = rows.glob(lr);
            if (i >= m_aug) break;
            const double yi = y[lr];
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
        double s = 0.0;
        if (warp == 0) {
#pragma unroll
            for (int w = 0; w < NW; ++w) s += red[w * IB_NB + lane];
        }
        if constexpr (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            double *buf = xc.xs + xc.flip * C * IB_NB;
            if (warp == 0)
                for (int r = 0; r < C; ++r) cl.map_shared_rank(buf, r)[rows.rank * IB_NB + lane] = s;
            cl.sync();
            if (warp == 0) {
                s = 0.0;
#pragma unroll
                for (int r = 0; r < C; ++r) s += buf[r * IB_NB + lane];
            }
            xc.flip ^= 1;
        }
        if (warp == 0) {
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
        for (int64_t lr = lr0 + tid;; lr += THREADS) {
            const int64_t i = rows.glob(lr);
            if (i >= m_aug) break;
            const int64_t li = i - k;
            const double *row = D.F + i + k * ld;
            double t = 0.0;
            if (li >= IB_NB) {
#pragma unroll
                for (int l = 0; l < IB_NB; ++l)
                    if (l < nc) t = fma(row[(int64_t)l * ld], wv[l], t);
            } else {
#pragma unroll
                for (int l = 0; l < IB_NB; ++l) {
                    const double v = (l >= nc || li < l) ? 0.0 : (li == l ? 1.0 : row[(int64_t)l * ld]);
                    t = fma(v, wv[l], t);
                }
            }
            y[lr] -= t;
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
            // the block's 32 reciprocals of the diagonal at once (one division per lane),
            // so that the sequential chain below is a multiply and an FMA per step
            const double rinv = 1.0 / ((lane < bw) ? F[(c0 + lane) + (c0 + lane) * ld] : 1.0);
            if (!transpose) {
#pragma unroll
                for (int c = 31; c >= 0; --c) {
                    if (c >= bw) continue;
                    double xc = 0.0;
                    if (lane == c) xc = xv * rinv;
                    xc = __shfl_sync(0xffffffffu, xc, c);
                    if (lane == c) xv = xc;
                    if (lane < c) xv = fma(-rr[c], xc, xv);
                }
            } else {
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    if (r >= bw) continue;
                    double xr = 0.0;
                    if (lane == r) xr = xv * rinv;
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

// One gradient evaluation of every instance: clusters of C CTAs take instances from the
// queue (rank 0 draws, the others read its draw); each rank holds its stripes of y.
template <int THREADS, int C>
__global__ void __launch_bounds__(THREADS)
k_inv_eval(const InvDesc *__restrict__ descs, const int *__restrict__ order, int n_inst,
           int *__restrict__ queue, int n_src, int64_t y_rows, int64_t n_max)
{
    constexpr int NW = THREADS / 32;
    extern __shared__ double ib_sm[];
    double *y = ib_sm;                          // [y_rows]: this rank's stripes
    double *xv = y + y_rows;                    // [n_max]   (rank 0)
    double *red = xv + n_max;                   // [NW][32]
    double *wv = red + NW * IB_NB;              // [32]
    double *gs = wv + IB_NB;                    // [IB_MAX_SENS]
    double *th = gs + IB_MAX_SENS;              // [4 IB_MAX_SRC]
    IbXchg xc;
    xc.xs = th + 4 * IB_MAX_SRC;                // [2][C][32]
    xc.xd = xc.xs + 2 * C * IB_NB;              // [C][4 IB_MAX_SRC]
    xc.flip = 0;
    __shared__ int s_q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    IbRows<C> rows;
    rows.rank = 0;
    if constexpr (C > 1) rows.rank = (int)cg::this_cluster().block_rank();
    const bool lead = rows.rank == 0;
    for (;;) {
        if (lead && tid == 0) s_q = atomicAdd(queue, 1);
        int q;
        if constexpr (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            q = *cl.map_shared_rank(&s_q, 0);
            cl.sync();                          // rank 0 keeps its shared memory until read
        } else {
            __syncthreads();
            q = s_q;
        }
        if (q >= n_inst) break;
        const InvDesc D = descs[order[q]];
        const int64_t n = D.n_feat;
        for (int t = tid; t < 4 * n_src; t += THREADS) th[t] = D.theta[t];
        __syncthreads();
        // source at the interior rows, zero elsewhere
        for (int64_t lr = tid;; lr += THREADS) {
            const int64_t i = rows.glob(lr);
            if (i >= D.m_aug) break;
            double v = 0.0;
            if (i < D.n_int) {
                const double px = D.x_int[2 * i], py = D.x_int[2 * i + 1];
                for (int s = 0; s < n_src; ++s) {
                    const double dx = px - th[4 * s], dy = py - th[4 * s + 1], w = th[4 * s + 2];
                    v += th[4 * s + 3] * exp(-(dx * dx + dy * dy) / (2.0 * w * w));
                }
            }
            y[lr] = v;
        }
        __syncthreads();
        ib_apply_q<THREADS, C>(D, rows, y, red, wv, xc, true);
        // (Q^T y)[0, n] to rank 0
        if constexpr (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            double *xv0 = cl.map_shared_rank(xv, 0);
            for (int64_t lr = tid;; lr += THREADS) {
                const int64_t i = rows.glob(lr);
                if (i >= n) break;
                xv0[i] = y[lr];
            }
            cl.sync();
        } else {
            for (int64_t j = tid; j < n; j += THREADS) xv[j] = y[j];
            __syncthreads();
        }
        if (lead) {
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
        }
        // z = Q [w; 0]
        {
            const double *w0 = xv;
            if constexpr (C > 1) {
                cg::cluster_group cl = cg::this_cluster();
                cl.sync();                                           // w complete on rank 0
                w0 = cl.map_shared_rank(xv, 0);
            }
            for (int64_t lr = tid;; lr += THREADS) {
                const int64_t i = rows.glob(lr);
                if (i >= D.m_aug) break;
                y[lr] = (i < n) ? w0[i] : 0.0;
            }
        }
        __syncthreads();
        ib_apply_q<THREADS, C>(D, rows, y, red, wv, xc, false);
        // dL/dtheta = sum over the interior rows of z_i ds(x_i)/dtheta
        double acc[4 * IB_MAX_SRC];
#pragma unroll
        for (int t = 0; t < 4 * IB_MAX_SRC; ++t) acc[t] = 0.0;
        for (int64_t lr = tid;; lr += THREADS) {
            const int64_t i = rows.glob(lr);
            if (i >= D.n_int) break;
            const double px = D.x_int[2 * i], py = D.x_int[2 * i + 1], zi = y[lr];
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
            if constexpr (C > 1) {
                if (tid == 0) *(cg::this_cluster().map_shared_rank(xc.xd, 0) + rows.rank * 4 * IB_MAX_SRC + t) = v;
            } else {
                if (tid == 0) D.dtheta[t] = v;
            }
        }
        if constexpr (C > 1) {
            cg::this_cluster().sync();
            if (lead)                                    // the ranks' sums in rank order
                for (int t = tid; t < 4 * n_src; t += THREADS) {
                    double v = 0.0;
                    for (int r = 0; r < C; ++r) v += xc.xd[r * 4 * IB_MAX_SRC + t];
                    D.dtheta[t] = v;
                }
        }
        __syncthreads();
    }
}

// The evaluation with the explicit thin Q of the interior rows, Qi = rows [0, n_int) of
// Q [I_n; 0] (n_int x n, kept by the plan): since y = [s; 0; 0] is zero below the
// interior rows and the gradient reads z on them only,
//   (Q^T y)[0, n] = Qi^T s      and      z[0, n_int) = (Q [w; 0])[0, n_int) = Qi w,
// 2 n_int n FP64 FMAs per evaluation instead of the reflectors' 4 m_aug n.  With a
// cluster, s is computed in row stripes and gathered into every rank, the columns of
// Qi^T s are dealt in groups of four over the ranks (results into rank 0), rank 0 runs
// the substitutions and the sensor products, and each rank forms z on its row stripes.
template <int THREADS, int C>
__global__ void __launch_bounds__(THREADS)
k_inv_eval_q(const InvDesc *__restrict__ descs, const int *__restrict__ order, int n_inst,
             int *__restrict__ queue, int n_src, int64_t nint_max, int64_t n_max)
{
    constexpr int NW = THREADS / 32;
    extern __shared__ double ib_sm[];
    double *sv = ib_sm;                         // [nint_max]  s at the interior rows
    double *xv = sv + nint_max;                 // [n_max]     Qi^T s, then w
    double *red = xv + n_max;                   // [NW][32]
    double *gs = red + NW * IB_NB;              // [IB_MAX_SENS]
    double *th = gs + IB_MAX_SENS;              // [4 IB_MAX_SRC]
    double *xd = th + 4 * IB_MAX_SRC;           // [C][4 IB_MAX_SRC]
    __shared__ int s_q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    IbRows<C> rows;
    rows.rank = 0;
    if constexpr (C > 1) rows.rank = (int)cg::this_cluster().block_rank();
    const bool lead = rows.rank == 0;
    for (;;) {
        if (lead && tid == 0) s_q = atomicAdd(queue, 1);
        int q;
        if constexpr (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            q = *cl.map_shared_rank(&s_q, 0);
            cl.sync();                          // rank 0 keeps its shared memory until read
        } else {
            __syncthreads();
            q = s_q;
        }
        if (q >= n_inst) break;
        const InvDesc D = descs[order[q]];
        const int64_t n = D.n_feat, n_int = D.n_int, ldq = D.ldq;
        const double *Qi = D.Q;
        for (int t = tid; t < 4 * n_src; t += THREADS) th[t] = D.theta[t];
        __syncthreads();
        // s at the interior rows (this rank's stripes), into every rank
        for (int64_t lr = tid;; lr += THREADS) {
            const int64_t i = rows.glob(lr);
            if (i >= n_int) break;
            const double px = D.x_int[2 * i], py = D.x_int[2 * i + 1];
            double v = 0.0;
            for (int s = 0; s < n_src; ++s) {
                const double dx = px - th[4 * s], dy = py - th[4 * s + 1], w = th[4 * s + 2];
                v += th[4 * s + 3] * exp(-(dx * dx + dy * dy) / (2.0 * w * w));
            }
            if constexpr (C > 1) {
                cg::cluster_group cl = cg::this_cluster();
                for (int r = 0; r < C; ++r) cl.map_shared_rank(sv, r)[i] = v;
            } else {
                sv[i] = v;
            }
        }
        if constexpr (C > 1) cg::this_cluster().sync();
        else __syncthreads();
        // t = Qi^T s: a warp per group of four columns, lanes over the rows (coalesced)
        {
            double *t_out = xv;
            if constexpr (C > 1) t_out = cg::this_cluster().map_shared_rank(xv, 0);
            const int64_t ngrp = (n + 3) / 4;
            for (int64_t g = rows.rank + (int64_t)C * warp; g < ngrp; g += (int64_t)C * NW) {
                const int64_t j0 = 4 * g;
                const int nc = (int)fl_min64(4, n - j0);
                const double *q0 = Qi + j0 * ldq;
                double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                if (nc == 4) {
#pragma unroll 4
                    for (int64_t i = lane; i < n_int; i += 32) {
                        const double si = sv[i];
                        a0 = fma(q0[i], si, a0);
                        a1 = fma(q0[i + ldq], si, a1);
                        a2 = fma(q0[i + 2 * ldq], si, a2);
                        a3 = fma(q0[i + 3 * ldq], si, a3);
                    }
                } else {
                    for (int64_t i = lane; i < n_int; i += 32) {
                        const double si = sv[i];
                        a0 = fma(q0[i], si, a0);
                        if (nc > 1) a1 = fma(q0[i + ldq], si, a1);
                        if (nc > 2) a2 = fma(q0[i + 2 * ldq], si, a2);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                    a3 += __shfl_xor_sync(0xffffffffu, a3, o);
                }
                if (lane < nc) t_out[j0 + lane] = (lane == 0) ? a0 : (lane == 1) ? a1 : (lane == 2) ? a2 : a3;
            }
        }
        if constexpr (C > 1) cg::this_cluster().sync();
        else __syncthreads();
        if (lead) {
            ib_trsv<THREADS>(D, xv, false);                          // beta
            for (int64_t j = tid; j < n; j += THREADS) D.beta[j] = xv[j];
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
            for (int64_t j = tid; j < n; j += THREADS) {
                double a = 0.0;
                for (int64_t s = 0; s < D.n_sens; ++s) a = fma(D.H[s * n + j], gs[s], a);
                xv[j] = a;
            }
            __syncthreads();
            ib_trsv<THREADS>(D, xv, true);                           // w
        }
        if constexpr (C > 1) {                                       // w into every rank
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            if (!lead) {
                const double *w0 = cl.map_shared_rank(xv, 0);
                for (int64_t j = tid; j < n; j += THREADS) xv[j] = w0[j];
            }
            __syncthreads();
        }
        // z_i = (Qi w)_i on this rank's row stripes, and dL/dtheta from it
        double acc[4 * IB_MAX_SRC];
#pragma unroll
        for (int t = 0; t < 4 * IB_MAX_SRC; ++t) acc[t] = 0.0;
        for (int64_t lr = tid;; lr += THREADS) {
            const int64_t i = rows.glob(lr);
            if (i >= n_int) break;
            const double *qr = Qi + i;
            double z0 = 0.0, z1 = 0.0, z2 = 0.0, z3 = 0.0;
            int64_t j = 0;
#pragma unroll 2
            for (; j + 4 <= n; j += 4) {
                z0 = fma(qr[j * ldq], xv[j], z0);
                z1 = fma(qr[(j + 1) * ldq], xv[j + 1], z1);
                z2 = fma(qr[(j + 2) * ldq], xv[j + 2], z2);
                z3 = fma(qr[(j + 3) * ldq], xv[j + 3], z3);
            }
            for (; j < n; ++j) z0 = fma(qr[j * ldq], xv[j], z0);
            const double zi = (z0 + z1) + (z2 + z3);
            const double px = D.x_int[2 * i], py = D.x_int[2 * i + 1];
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
            if constexpr (C > 1) {
                if (tid == 0) *(cg::this_cluster().map_shared_rank(xd, 0) + rows.rank * 4 * IB_MAX_SRC + t) = v;
            } else {
                if (tid == 0) D.dtheta[t] = v;
            }
        }
        if constexpr (C > 1) {
            cg::this_cluster().sync();
            if (lead)                                    // the ranks' sums in rank order
                for (int t = tid; t < 4 * n_src; t += THREADS) {
                    double v = 0.0;
                    for (int r = 0; r < C; ++r) v += xd[r * 4 * IB_MAX_SRC + t];
                    D.dtheta[t] = v;
                }
        }
        __syncthreads();
    }
}

size_t ib_q_smem(int threads, int64_t nint_max, int64_t n_max, int cluster)
{
    return sizeof(double) * ((size_t)nint_max + (size_t)n_max + (size_t)(threads / 32) * IB_NB + IB_MAX_SENS +
                             4 * IB_MAX_SRC + (size_t)cluster * 4 * IB_MAX_SRC);
}

// rows of y one rank holds: its stripes of the tallest instance
int64_t ib_rows(int64_t m_aug_max, int cluster)
{
    return 32 * ((fl_cdiv(m_aug_max, 32) + cluster - 1) / cluster);
}

size_t ib_smem(int threads, int64_t m_aug_max, int64_t n_max, int cluster)
{
    return sizeof(double) * ((size_t)ib_rows(m_aug_max, cluster) + (size_t)n_max + (size_t)(threads / 32) * IB_NB +
                             IB_NB + IB_MAX_SENS + 4 * IB_MAX_SRC + 2 * (size_t)cluster * IB_NB +
                             (size_t)cluster * 4 * IB_MAX_SRC);
}

}  // namespace

struct fastlsq_inverse_plan {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_inst = 0, n_src = 0;
    int64_t m_aug_max = 0, n_max = 0, nint_max = 0;
    int thin_q = 0;               // evaluations use the explicit thin Q of the interior rows
    std::vector<fastlsq_factor *> factors;
    std::vector<double *> Qbuf;   // thin-Q form: per instance rows [0, n_int) of Q [I; 0]
    double *H = nullptr;          // sensor matrices, all instances
    InvDesc *d_desc = nullptr;
    int *d_order = nullptr;
    int *d_queue = nullptr;
    std::vector<InvDesc> h_desc;
    std::vector<int> h_order;
};

namespace {

template <int THREADS, int C>
cudaError_t ib_launch(const fastlsq_inverse_plan *P, cudaStream_t st, int grid, size_t smem)
{
    static FlOncePerDevice once;
    if (once.pending(P->device)) {
        // the largest the device allows, so that a later plan with taller instances fits
        int optin = 0;
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_inv_eval<THREADS, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_inv_eval_q<THREADS, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - 1024);
        if (e != cudaSuccess) return e;
        once.done(P->device);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (P->thin_q)
        return cudaLaunchKernelEx(&cfg, k_inv_eval_q<THREADS, C>, (const InvDesc *)P->d_desc,
                                  (const int *)P->d_order, P->n_inst, P->d_queue, P->n_src, P->nint_max, P->n_max);
    return cudaLaunchKernelEx(&cfg, k_inv_eval<THREADS, C>, (const InvDesc *)P->d_desc, (const int *)P->d_order,
                              P->n_inst, P->d_queue, P->n_src, ib_rows(P->m_aug_max, C), P->n_max);
}

void plan_free(fastlsq_inverse_plan *P)
{
    if (!P) return;
    for (fastlsq_factor *f : P->factors) fastlsq_factor_destroy(f);
    for (double *q : P->Qbuf)
        if (q) cudaFreeAsync(q, P->stream);
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
    int64_t m_max = 0, n_max = 0, maug_max = 0, nint_max = 0;
    for (int q = 0; q < n_inst; ++q) {
        const fastlsq_inverse_instance &I = inst[q];
        if (I.n_int < 1 || I.n_bc < 0 || I.n_feat < 1 || I.n_feat > FL_MAX_FEAT || I.n_sens < 1 ||
            I.n_sens > IB_MAX_SENS || !I.x_int || (I.n_bc && !I.x_bc) || !I.W || !I.b || !I.sensors || !I.y_obs ||
            !I.theta || !I.beta || !I.loss || !I.dtheta)
            return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_prepare: bad instance %d", q);
        m_max = std::max<int64_t>(m_max, fl_round_up(I.n_int + I.n_bc, 4));
        n_max = std::max<int64_t>(n_max, I.n_feat);
        maug_max = std::max<int64_t>(maug_max, I.n_int + I.n_bc + I.n_feat);
        nint_max = std::max<int64_t>(nint_max, I.n_int);
    }
    // the evaluation keeps y [m_aug] (split over a cluster's ranks; thin-Q form: s at the
    // interior rows) and one n-vector per CTA in shared memory: the plan must fit at
    // least the smallest configuration
    const int thin_q = ctx->inverse_thin_q;
    if ((thin_q ? ib_q_smem(256, nint_max, n_max, 4) : ib_smem(256, maug_max, n_max, 4)) >
        (size_t)ctx->max_smem_optin - 1024)
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
    P->nint_max = nint_max;
    P->thin_q = thin_q;
    P->factors.assign(n_inst, nullptr);
    P->Qbuf.assign(n_inst, nullptr);
    P->h_desc.resize(n_inst);
    size_t h_total = 0;
    for (int q = 0; q < n_inst; ++q) h_total += (size_t)inst[q].n_sens * inst[q].n_feat;
    cudaError_t e = cudaMallocAsync(&P->H, sizeof(double) * h_total, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P->d_desc, sizeof(InvDesc) * n_inst, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P->d_order, sizeof(int) * n_inst, ctx->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&P->d_queue, sizeof(int), ctx->stream);
    int rc = (e == cudaSuccess) ? 0 : fl_cuda(ctx, e, "inverse_prepare buffers");
    size_t h_off = 0;
    std::vector<size_t> h_at(n_inst);
    for (int q = 0; q < n_inst; ++q) {
        h_at[q] = h_off;
        h_off += (size_t)inst[q].n_sens * inst[q].n_feat;
    }
    // The factorisations are independent: they are spread over a few worker contexts,
    // each on a stream of its own, so that the panel chains of small instances (which
    // leave most SMs idle) overlap.  Instances go to the worker with the least work so
    // far, largest first (m n^2 each), so every worker's workspace reaches its size on
    // its first instance.  Each worker has its own operator and prefactor buffers.
    struct Worker {
        fastlsq_ctx *c = nullptr;
        cudaStream_t s = nullptr;
        double *A64 = nullptr, *pref = nullptr;
        std::vector<int> todo;
        double load = 0.0;
    };
    const int n_work = std::min<int>(IB_SETUP_WORKERS, n_inst);
    std::vector<Worker> wk(n_work);
    {
        std::vector<int> by_cost(n_inst);
        std::iota(by_cost.begin(), by_cost.end(), 0);
        auto cost = [&](int q) {
            return (double)(inst[q].n_int + inst[q].n_bc + inst[q].n_feat) * (double)inst[q].n_feat *
                   (double)inst[q].n_feat;
        };
        std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return cost(a) > cost(b); });
        for (int q : by_cost) {
            Worker *lo = &wk[0];
            for (Worker &w : wk)
                if (w.load < lo->load) lo = &w;
            lo->todo.push_back(q);
            lo->load += cost(q);
        }
    }
    cudaEvent_t ready = nullptr;
    if (rc >= 0) {
        e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ready, ctx->stream);     // inputs and P->H
        if (e != cudaSuccess) rc = fl_cuda(ctx, e, "inverse_prepare event");
    }
    for (Worker &w : wk) {
        if (rc < 0) break;
        e = cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            rc = fl_cuda(ctx, e, "inverse_prepare stream");
            break;
        }
        const int crc = fastlsq_create(&w.c, ctx->device, (void *)w.s);
        if (crc < 0) {
            rc = fl_fail(ctx, crc, "inverse_prepare: worker context");
            break;
        }
        w.c->panel_reg = ctx->panel_reg;
        w.c->row_panel = ctx->row_panel;
        w.c->lookahead = ctx->lookahead;
        w.c->fuse_next = ctx->fuse_next;
        w.c->split_rows = ctx->split_rows;
        e = cudaStreamWaitEvent(w.s, ready, 0);
        if (e == cudaSuccess) e = cudaMallocAsync(&w.A64, sizeof(double) * m_max * n_max, w.s);
        if (e == cudaSuccess) e = cudaMallocAsync(&w.pref, sizeof(double) * (2 + FL_MAX_PP) * n_max, w.s);
        if (e != cudaSuccess) rc = fl_cuda(ctx, e, "inverse_prepare worker buffers");
    }
    // issue round-robin over the workers (the host never waits inside the loop)
    for (size_t r = 0; rc >= 0; ++r) {
        bool any = false;
        for (Worker &w : wk) {
            if (rc < 0 || r >= w.todo.size()) continue;
            any = true;
            const int q = w.todo[r];
            fastlsq_ctx *c = w.c;
            const fastlsq_inverse_instance &I = inst[q];
            const int64_t n = I.n_feat, m = I.n_int + I.n_bc, ld = fl_round_up(m, 4);
            const double scale = 1.0 / sqrt((double)n);
            double *A64 = w.A64, *pref = w.pref;
            int wrc = 0;
            do {
                if ((wrc = fl_prefactors(c, opL, I.W, n, scale, 1.0, pref)) < 0) break;
                if ((wrc = fl_launch_assemble_f64(c, opL, I.x_int, I.n_int, I.W, I.b, n, pref, A64, ld, 0,
                                                  1.0)) < 0) break;
                if (I.n_bc) {
                    if ((wrc = fl_prefactors(c, opI, I.W, n, scale, o->bc_weight, pref)) < 0) break;
                    if ((wrc = fl_launch_assemble_f64(c, opI, I.x_bc, I.n_bc, I.W, I.b, n, pref, A64, ld, I.n_int,
                                                      o->bc_weight)) < 0) break;
                }
                wrc = fastlsq_lstsq(c, FASTLSQ_PREC_FP64, A64, FASTLSQ_F64, ld, m, n, o->mu, nullptr, 0, ld, nullptr,
                                    n, nullptr, 0, 0, FASTLSQ_REFINE_CLASSICAL, 0.0, &P->factors[q], nullptr);
                if (wrc < 0) break;
                double *H = P->H + h_at[q];
                k_sensor_matrix<<<dim3((unsigned)fl_cdiv(n, 256), (unsigned)I.n_sens), 256, 0, w.s>>>(
                    I.sensors, I.n_sens, I.W, I.b, n, scale, H);
                if (cudaGetLastError() != cudaSuccess) {
                    wrc = fl_fail(c, FASTLSQ_ERR_CUDA, "sensor matrix");
                    break;
                }
                const fastlsq_factor *f = P->factors[q];
                // thin-Q form: Q [I; 0] into a copy of the factor's storage with n more
                // columns, then its interior rows kept (ldq rows, a multiple of 4)
                const int64_t ldq = fl_round_up(I.n_int, 4);
                if (thin_q) {
                    double *G = nullptr;
                    cudaError_t ge = cudaMallocAsync(&G, sizeof(double) * f->ld * 2 * n, w.s);
                    if (ge == cudaSuccess)
                        ge = cudaMemcpyAsync(G, f->F, sizeof(double) * f->ld * n, cudaMemcpyDeviceToDevice, w.s);
                    if (ge != cudaSuccess) {
                        if (G) cudaFreeAsync(G, w.s);
                        wrc = fl_cuda(c, ge, "thin Q buffer");
                        break;
                    }
                    wrc = fl_form_q_f64(c, G, f->ld, f->m_aug, n, f->nb, (const double *)f->T, n);
                    if (wrc >= 0) {
                        ge = cudaMallocAsync(&P->Qbuf[q], sizeof(double) * ldq * n, w.s);
                        if (ge == cudaSuccess) ge = cudaMemsetAsync(P->Qbuf[q], 0, sizeof(double) * ldq * n, w.s);
                        if (ge == cudaSuccess)
                            ge = cudaMemcpy2DAsync(P->Qbuf[q], sizeof(double) * ldq, G + n * f->ld,
                                                   sizeof(double) * f->ld, sizeof(double) * I.n_int, n,
                                                   cudaMemcpyDeviceToDevice, w.s);
                        if (ge != cudaSuccess) wrc = fl_cuda(c, ge, "thin Q copy");
                    }
                    cudaFreeAsync(G, w.s);
                    if (wrc < 0) break;
                }
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
                D.Q = P->Qbuf[q];
                D.ldq = ldq;
                D.beta = I.beta;
                D.loss = I.loss;
                D.dtheta = I.dtheta;
            } while (0);
            if (wrc < 0) rc = fl_fail(ctx, wrc, "inverse_prepare: instance %d: %s", q, c->last_error.c_str());
        }
        if (!any) break;
    }
    // join the workers: their kernels' error flags, then their buffers; the kept factors
    // move to the plan's stream (their memory is stream-ordered and complete here)
    for (Worker &w : wk) {
        if (w.c) {
            const int src = fastlsq_sync(w.c);
            if (src < 0 && rc >= 0) rc = fl_fail(ctx, src, "inverse_prepare: %s", w.c->last_error.c_str());
        }
        if (w.A64) cudaFreeAsync(w.A64, w.s);
        if (w.pref) cudaFreeAsync(w.pref, w.s);
        if (w.s) cudaStreamSynchronize(w.s);
    }
    for (fastlsq_factor *f : P->factors) {
        if (!f) continue;
        f->ctx = ctx;
        f->stream = ctx->stream;
    }
    for (Worker &w : wk) {
        if (w.c) fastlsq_destroy(w.c);
        if (w.s) cudaStreamDestroy(w.s);
    }
    if (ready) cudaEventDestroy(ready);
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
                                    int32_t ctas_per_sm, int32_t cluster)
{
    if (!ctx || !P) return FASTLSQ_ERR_INVALID;
    if ((threads != 256 && threads != 512) || ctas_per_sm < 1 || ctas_per_sm > 4 ||
        (cluster != 1 && cluster != 2 && cluster != 4))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID,
                       "inverse_eval: threads 256 or 512, 1..4 CTAs per SM, clusters of 1, 2 or 4");
    const size_t smem = P->thin_q ? ib_q_smem(threads, P->nint_max, P->n_max, cluster)
                                  : ib_smem(threads, P->m_aug_max, P->n_max, cluster);
    if (smem * ctas_per_sm > (size_t)ctx->max_smem_optin)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "inverse_eval: %d CTAs per SM do not fit in shared memory",
                       ctas_per_sm);
    // one cluster per instance at most; whole clusters only
    const int clusters = std::max(1, std::min<int>(P->n_inst, ctx->num_sms * ctas_per_sm / cluster));
    const int grid = clusters * cluster;
    cudaError_t e = cudaMemsetAsync(P->d_queue, 0, sizeof(int), ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "inverse_eval queue");
    FL_PROF(ctx, FASTLSQ_K_ADJOINT);
    if (threads == 256)
        e = (cluster == 1)   ? ib_launch<256, 1>(P, ctx->stream, grid, smem)
            : (cluster == 2) ? ib_launch<256, 2>(P, ctx->stream, grid, smem)
                             : ib_launch<256, 4>(P, ctx->stream, grid, smem);
    else
        e = (cluster == 1)   ? ib_launch<512, 1>(P, ctx->stream, grid, smem)
            : (cluster == 2) ? ib_launch<512, 2>(P, ctx->stream, grid, smem)
                             : ib_launch<512, 4>(P, ctx->stream, grid, smem);
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

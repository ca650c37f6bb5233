// Blocked Householder QR and the solves built on it (Sec. 2.3: "beta* = A^+ b
// via QR"; Sec. 2.4: Tikhonov rows sqrt(mu) I; Sec. 3.8: pre-factored solves).
//
// Layout: the factor F is column-major (ld), rows [0, m_aug), columns [0, n)
// hold the matrix, columns [n, n + nrhs) hold right-hand sides that ride along
// with the trailing updates (so Q^T b comes out of the factorisation).  After
// factorisation F holds R on and above the diagonal and the Householder vectors
// (unit diagonal implied) below it; tau[j] are the reflector scalars and, per
// panel p of width NB, T_p is the upper-triangular NB x NB matrix of the compact
// WY form H_k ... H_{k+NB-1} = I - V T V^T.
//
// Reflector convention (as LAPACK): beta = -sign(a_jj) ||a_j(j:)||,
// tau = (beta - a_jj) / beta, v = a_j(j+1:) / (a_jj - beta), v_j = 1.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "gridsync.cuh"
#include "qr.cuh"
#include "trail_z.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int PANEL_THREADS = 1024;
constexpr int PANEL_WARPS = PANEL_THREADS / 32;
constexpr int APPLY_THREADS = 512;
constexpr int CL_MAX = 16;

template <typename T> __device__ __forceinline__ T fl_sqrt(T v);
template <> __device__ __forceinline__ float fl_sqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double fl_sqrt<double>(double v) { return sqrt(v); }

template <typename T> __device__ __forceinline__ bool fl_isfinite(T v) { return isfinite(v); }

__device__ __forceinline__ void raise_flag(int *flag, int code)
{
    if (flag) atomicCAS(flag, 0, code);
}

template <typename T, int NB>
struct PanelSmem {
    static constexpr int LD = NB + 1;   // padded row stride of the panel slice
    static size_t bytes(int rpc)
    {
        return sizeof(T) * ((size_t)rpc * LD + PANEL_WARPS * 33 + 2 * (CL_MAX + 1) * NB +
                            2 * NB * (NB + 1) + NB);
    }
};

// Panel factorisation on a cluster of CL CTAs.  CTA `rank` owns panel rows
// [rank * rpc, min((rank+1) * rpc, mp)) in shared memory; rpc >= ncols so rank 0
// owns every diagonal row.  For each column j one cluster-wide exchange (DSMEM
// stores + one cluster barrier) delivers: the dot products of column j with
// every column l > j below the diagonal (sum over rows i > j of a_ij a_il), the
// diagonal row a_j., and the Gram entries v_l^T v_{j-1} (l < j-1) that the
// compact-WY recurrence T(0:c, c) = -tau_c T(0:c, 0:c) V(:, 0:c)^T v_c needs
// (T is formed once at the end).  The update pass that applies H_j to the rows
// also accumulates the next column's dots and this column's Gram entries, so a
// column costs one pass over the slice; each thread updates four independent
// rows per iteration and the two rows next to the diagonal are handled apart.
template <typename T, int NB>
__global__ void __launch_bounds__(PANEL_THREADS, 1)
k_panel(T *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols, int rpc,
        T *__restrict__ tau_out, T *__restrict__ T_out, int *flag)
{
    constexpr int LDP = PanelSmem<T, NB>::LD;
    constexpr int RPW = 32 / NB;                 // rows per warp step
    constexpr int RSTEP = PANEL_WARPS * RPW;     // rows per block step
    constexpr int U = 4;                         // rows per thread per iteration
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *P = reinterpret_cast<T *>(smem_raw);
    T *red = P + (size_t)rpc * LDP;                 // [PANEL_WARPS][33]
    T *xbuf = red + PANEL_WARPS * 33;               // [2][CL_MAX + 1][NB]
    T *Tm = xbuf + 2 * (CL_MAX + 1) * NB;           // [NB][NB + 1] T(row, col)
    T *G = Tm + NB * (NB + 1);                      // [NB][NB + 1] G(q, c) = v_q^T v_c
    T *tauv = G + NB * (NB + 1);                    // [NB]

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int CL = (int)cluster.num_blocks();
    const int64_t mp = m - k;
    const int64_t c0 = (int64_t)rank * rpc;
    const int nown = (int)fl_max64(0, fl_min64(rpc, mp - c0));
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int l = lane % NB;       // column handled by this lane
    const int sub = lane / NB;     // row sub-slot within the warp step
    const int rb0 = warp * RPW + sub;
    const unsigned FULL = 0xffffffffu;

    for (int idx = threadIdx.x; idx < nown * NB; idx += PANEL_THREADS) {
        int c = idx / nown, r = idx % nown;
        P[r * LDP + c] = (c < ncols) ? F[(k + c0 + r) + (k + c) * ld] : T(0);
    }
    for (int idx = threadIdx.x; idx < 2 * NB * (NB + 1); idx += PANEL_THREADS) Tm[idx] = T(0);
    __syncthreads();

    // dots of column 0 with every column, rows i > 0
    T acc = T(0);
    for (int r = rb0; r < nown; r += RSTEP)
        if (c0 + r > 0) acc += P[r * LDP] * P[r * LDP + l];

    for (int j = 0; j <= ncols; ++j) {
        const int par = j & 1;
        // block reduction, transposed: warp c sums column c over the 32 warps (and
        // row sub-slots), then its lane 0 sends the CTA's partial to every rank
        red[warp * 33 + lane] = acc;
        __syncthreads();
        if (warp < NB) {
            T part = T(0);
#pragma unroll
            for (int s = 0; s < RPW; ++s) part += red[lane * 33 + s * NB + warp];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
            if (lane < CL) {
                T *rb = cluster.map_shared_rank(xbuf, lane);
                rb[(par * (CL_MAX + 1) + rank) * NB + warp] = part;
                if (rank == 0) rb[(par * (CL_MAX + 1) + CL_MAX) * NB + warp] =
                    (j < ncols) ? P[j * LDP + warp] : T(0);
            }
        }
        cluster.sync();
        const T *xb = xbuf + par * (CL_MAX + 1) * NB;
        // cross-CTA sums: four interleaved chains, the same order on every rank
        T d0 = T(0), d1 = T(0), d2 = T(0), d3 = T(0);
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        const int jc = (j < ncols) ? j : 0;
        for (int q = 0; q < CL; q += 4) {
            d0 += xb[q * NB + l];
            s0 += xb[q * NB + jc];
            if (q + 1 < CL) { d1 += xb[(q + 1) * NB + l]; s1 += xb[(q + 1) * NB + jc]; }
            if (q + 2 < CL) { d2 += xb[(q + 2) * NB + l]; s2 += xb[(q + 2) * NB + jc]; }
            if (q + 3 < CL) { d3 += xb[(q + 3) * NB + l]; s3 += xb[(q + 3) * NB + jc]; }
        }
        const T dl = (d0 + d1) + (d2 + d3);
        const T ssum = (s0 + s1) + (s2 + s3);
        // Gram column j-1 (lanes l < j-1), kept for the T recurrence at the end
        if (j >= 1 && warp == 0 && lane < NB && rank == 0 && l < j - 1) G[l * (NB + 1) + (j - 1)] = dl;
        if (j == ncols) break;

        // reflector for column j (every thread computes the same scalars)
        const T ss = ssum;
        const T ajj = xb[CL_MAX * NB + j];
        const T topl = xb[CL_MAX * NB + l];
        T beta = ajj, tauj = T(0), inv = T(0);
        if (!fl_isfinite(ss) || !fl_isfinite(ajj)) {
            raise_flag(flag, FL_DEVERR_NONFINITE);
        } else if (ss > T(0)) {
            T nrm = fl_sqrt<T>(ajj * ajj + ss);
            beta = (ajj >= T(0)) ? -nrm : nrm;
            tauj = (beta - ajj) / beta;
            inv = T(1) / (ajj - beta);
        }
        const T wl = (l > j) ? tauj * (topl + inv * dl) : T(0);
        if (threadIdx.x == 0) tauv[j] = tauj;
        const int jn = (j + 1) % NB;

        // apply H_j to the owned rows below j+1: next-column dots (l > j) and Gram
        // entries v_l^T v_j (l < j); U independent rows per iteration
        acc = T(0);
        for (int r0 = rb0 - sub; r0 < nown; r0 += U * RSTEP) {      // warp-uniform bound
            T pj[U], pl[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + sub + u * RSTEP;
                ok[u] = (r < nown) && (c0 + r > j + 1);
                pj[u] = ok[u] ? P[r * LDP + j] : T(0);
                pl[u] = ok[u] ? P[r * LDP + l] : T(0);
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + sub + u * RSTEP;
                const T vj = pj[u] * inv;
                const T nl = (l > j) ? pl[u] - wl * vj : pl[u];
                if (ok[u]) P[r * LDP + l] = (l == j) ? vj : nl;
                const T nxt = __shfl_sync(FULL, nl, sub * NB + jn);
                const T add = (l < j) ? pl[u] * vj : ((l > j) ? nxt * nl : T(0));
                acc += ok[u] ? add : T(0);
            }
        }
        // the diagonal row j and the next row j + 1, on the rank that owns each
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int64_t g = j + q;                         // panel-local row
            const int r = (int)(g - c0);
            if (g >= mp || g >= ncols + 1 || r < 0 || r >= nown) continue;   // uniform per CTA
            if (warp != (r % RSTEP) / RPW) continue;        // owner warp (uniform)
            const bool mine = (sub == (r % RSTEP) % RPW);
            T pj = mine ? P[r * LDP + j] : T(0);
            T pl = mine ? P[r * LDP + l] : T(0);
            __syncwarp();
            if (mine) {
                if (q == 0) {                     // diagonal row: H_j maps it to (beta, a - w)
                    if (l > j) P[r * LDP + l] = pl - wl;
                    if (l == j) P[r * LDP + j] = beta;
                    if (l < j) acc += pl;         // v_j has a unit entry in row j
                } else {                          // row j + 1: update, Gram only
                    const T vj = pj * inv;
                    if (l > j) P[r * LDP + l] = pl - wl * vj;
                    if (l == j) P[r * LDP + j] = vj;
                    if (l < j) acc += pl * vj;
                }
            }
        }
    }

    // write back the slice; rank 0 forms T and writes tau, T
    __syncthreads();
    for (int idx = threadIdx.x; idx < nown * NB; idx += PANEL_THREADS) {
        int c = idx / nown, r = idx % nown;
        if (c < ncols) F[(k + c0 + r) + (k + c) * ld] = P[r * LDP + c];
    }
    if (rank == 0 && warp == 0) {
        // T(c, c) = tau_c ; T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c)   (lane = row)
        for (int c = 0; c < ncols; ++c) {
            const T tc = tauv[c];
            T sum = T(0);
            if (lane < c)
                for (int q = lane; q < c; ++q) sum += Tm[lane * (NB + 1) + q] * G[q * (NB + 1) + c];
            __syncwarp();
            if (lane < c) Tm[lane * (NB + 1) + c] = -tc * sum;
            if (lane == c) Tm[c * (NB + 1) + c] = tc;
            __syncwarp();
        }
        for (int idx = lane; idx < NB; idx += 32) tau_out[idx] = (idx < ncols) ? tauv[idx] : T(0);
        for (int idx = lane; idx < NB * NB; idx += 32) {
            int col = idx / NB, row = idx % NB;
            T_out[idx] = (col < ncols && row < ncols) ? Tm[row * (NB + 1) + col] : T(0);
        }
    }
}

// V(i, l) for panel-local row i of panel starting at column k (unit lower trapezoid)
template <typename T>
__device__ __forceinline__ T v_at(const T *__restrict__ F, int64_t ld, int64_t k, int64_t i,
                                  int l, int ncols)
{
    if (l >= ncols || i < l) return T(0);
    if (i == l) return T(1);
    return F[(k + i) + (k + l) * ld];
}

// Trailing update C -= V (T^T (V^T C)) of one panel (C: the columns right of the
// panel, right-hand sides included), in two kernels:
//  * k_trail_y: Y partials over row splits, Ypart[s][l][c] = sum over the rows of
//    split s of V(i,l) C(i,c); CTA tile = all NB rows of Y x TY_COLS columns, rows
//    streamed in chunks of TY_ROWS.  Chunks are read as 4-row vectors along the
//    columns of F (coalesced) into registers one chunk ahead of the one being
//    multiplied from shared memory.  The last CTA of a column tile forms Z = T^T Y.
//  * k_trail_c: C -= V Z on TC_ROWS x TC_COLS tiles; the tile of C is requested
//    first so its loads overlap the staging of V and Z.
// Rows past the end of the panel (up to the factor's 4-row padding) are zero in F,
// so 4-row vectors never need masking below row m_aug.
constexpr int TY_COLS = 128;
constexpr int TY_ROWS = 32;
constexpr int TY_THREADS = 256;

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

template <typename T>
__device__ __forceinline__ typename Vec4<T>::type v4_zero()
{
    typename Vec4<T>::type z;
    z.x = z.y = z.z = z.w = T(0);
    return z;
}

// V(i..i+3, l) as a vector, with the unit-lower-trapezoid mask on the top rows
template <typename T>
__device__ __forceinline__ typename Vec4<T>::type v_quad(const T *__restrict__ F, int64_t ld, int64_t k,
                                                          int64_t i, int l, int ncols)
{
    using V4 = typename Vec4<T>::type;
    if (l >= ncols) return v4_zero<T>();
    V4 v = *reinterpret_cast<const V4 *>(F + (k + i) + (k + l) * ld);
    if (i <= l) {                       // rows at or above the diagonal of column l
        v.x = (i + 0 < l) ? T(0) : (i + 0 == l ? T(1) : v.x);
        v.y = (i + 1 < l) ? T(0) : (i + 1 == l ? T(1) : v.y);
        v.z = (i + 2 < l) ? T(0) : (i + 2 == l ? T(1) : v.z);
        v.w = (i + 3 < l) ? T(0) : (i + 3 == l ? T(1) : v.w);
    }
    return v;
}

template <typename T, int NB>
struct TrailYSmem {
    // row-major chunks: C [TY_ROWS][TY_COLS + 4], V [TY_ROWS][NB + 4]
    static constexpr int CLD = TY_COLS + 4, VLD = NB + 4;
    static constexpr size_t stage = sizeof(T) * (size_t)TY_ROWS * (CLD + VLD);
    static constexpr size_t zscr = sizeof(T) * (size_t)(NB * TY_COLS + NB * NB);
    static constexpr size_t bytes = stage > zscr ? stage : zscr;
};

template <typename T, int NB, bool TFWD = false>
__global__ void __launch_bounds__(TY_THREADS)
k_trail_y(const T *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols, int64_t nct, int64_t coff,
          int64_t rows_per_split, T *__restrict__ Ypart, T *__restrict__ Z, const T *__restrict__ Tblk,
          int *__restrict__ counters)
{
    using V4 = typename Vec4<T>::type;
    constexpr int CLD = TrailYSmem<T, NB>::CLD, VLD = TrailYSmem<T, NB>::VLD;
    constexpr int NW = TY_THREADS / 32;              // warps
    constexpr int LPW = NB / NW;                     // l per warp (4 for NB = 32, 2 for 16, 1 for 8)
    constexpr int QPC = TY_ROWS / 4;                 // 4-row quads per chunk column
    constexpr int CQ = TY_COLS * QPC / TY_THREADS;   // C quads per thread per chunk
    static_assert(LPW >= 1 && CQ >= 1 && TY_COLS == 4 * 32, "tile");
    extern __shared__ __align__(16) unsigned char ty_raw[];
    T *sC = reinterpret_cast<T *>(ty_raw);           // [TY_ROWS][CLD]
    T *sV = sC + TY_ROWS * CLD;                      // [TY_ROWS][VLD]
    const int64_t mp = m - k;
    const int64_t cbase = (int64_t)blockIdx.x * TY_COLS;
    const int64_t rs0 = (int64_t)blockIdx.y * rows_per_split;
    const int64_t rs1 = fl_min64(mp, rs0 + rows_per_split);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lq = tid % QPC;                         // loader: quad within the chunk
    const int lc = tid / QPC;                         // loader: column (plus pass * 32)
    V4 rc[CQ], rv;

    auto load = [&](int64_t r0) {
        const int64_t i = r0 + 4 * lq;
#pragma unroll
        for (int ps = 0; ps < CQ; ++ps) {
            const int64_t c = cbase + lc + ps * (TY_THREADS / QPC);
            rc[ps] = (i < rs1 && c < nct) ? *reinterpret_cast<const V4 *>(F + (k + i) + (k + ncols + coff + c) * ld)
                                         : v4_zero<T>();
        }
        rv = (lc < NB && i < rs1) ? v_quad(F, ld, k, i, lc, ncols) : v4_zero<T>();
    };
    // 4-row vectors of one column land in 4 rows of the row-major chunk
    auto store = [&]() {
#pragma unroll
        for (int ps = 0; ps < CQ; ++ps) {
            T *d = sC + (4 * lq) * CLD + lc + ps * (TY_THREADS / QPC);
            d[0] = rc[ps].x;
            d[CLD] = rc[ps].y;
            d[2 * CLD] = rc[ps].z;
            d[3 * CLD] = rc[ps].w;
        }
        if (lc < NB) {
            T *d = sV + (4 * lq) * VLD + lc;
            d[0] = rv.x;
            d[VLD] = rv.y;
            d[2 * VLD] = rv.z;
            d[3 * VLD] = rv.w;
        }
    };

    // warp w owns l = LPW w .. LPW w + LPW - 1 (one broadcast read per row), lane owns
    // columns 4 lane .. 4 lane + 3 (one conflict-free 16-byte read per row)
    T acc[LPW][4];
#pragma unroll
    for (int a = 0; a < LPW; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);

    // two-level sum: each chunk's 32 rows into a fresh partial, the partials into acc,
    // so a split of many rows is not one long chain of roundings
    if (rs0 < rs1) load(rs0);
    for (int64_t r0 = rs0; r0 < rs1; r0 += TY_ROWS) {
        store();
        __syncthreads();
        if (r0 + TY_ROWS < rs1) load(r0 + TY_ROWS);          // next chunk in flight
        T cacc[LPW][4];
#pragma unroll
        for (int a = 0; a < LPW; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) cacc[a][b] = T(0);
#pragma unroll 8
        for (int r = 0; r < TY_ROWS; ++r) {
            const V4 cv = *reinterpret_cast<const V4 *>(sC + r * CLD + 4 * lane);
            T vl[LPW];
#pragma unroll
            for (int a = 0; a < LPW; ++a) vl[a] = sV[r * VLD + LPW * warp + a];
#pragma unroll
            for (int a = 0; a < LPW; ++a) {
                cacc[a][0] += vl[a] * cv.x;
                cacc[a][1] += vl[a] * cv.y;
                cacc[a][2] += vl[a] * cv.z;
                cacc[a][3] += vl[a] * cv.w;
            }
        }
#pragma unroll
        for (int a = 0; a < LPW; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += cacc[a][b];
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < LPW; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t c = cbase + 4 * lane + b;
            if (c < nct) Ypart[((int64_t)blockIdx.y * NB + LPW * warp + a) * nct + c] = acc[a][b];
        }
    int *cnt = counters + (int64_t)blockIdx.x * TREE_STRIDE;
    trail_finish_z<T, NB, TY_COLS, TY_THREADS, false, TFWD>(Ypart, (int)gridDim.y, nct, cbase, Tblk, Z, cnt,
                                                            cnt + 1, reinterpret_cast<T *>(ty_raw));
}

// C(i, c) -= sum_l V(i, l) Z(l, c).  CTA tile TC_ROWS x TC_COLS; each thread owns 4
// consecutive rows x 8 columns and reads and writes C as 4-row vectors.
constexpr int TC_ROWS = 128;
constexpr int TC_COLS = 64;

template <typename T, int NB>
__global__ void __launch_bounds__(256)
k_trail_c(T *__restrict__ F, int64_t ld, int64_t k, int64_t m, int ncols, int64_t nct, int64_t coff,
          const T *__restrict__ Z)
{
    using V4 = typename Vec4<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*sZ)[TC_COLS] = reinterpret_cast<T (*)[TC_COLS]>(smem_raw);                                // [NB][TC_COLS]
    T (*sV)[TC_ROWS] = reinterpret_cast<T (*)[TC_ROWS]>(smem_raw + sizeof(T) * NB * TC_COLS);    // [NB][TC_ROWS]
    const int64_t mp = m - k;
    const int64_t rbase = (int64_t)blockIdx.x * TC_ROWS;
    const int64_t cbase = (int64_t)blockIdx.y * TC_COLS;
    const int r4 = (threadIdx.x & 31) * 4;     // 4 consecutive rows
    const int c8 = (threadIdx.x >> 5) * 8;     // 8 columns
    const int64_t i0 = rbase + r4;
    // the thread's C tile first: its loads overlap the staging below
    V4 cur[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int64_t c = cbase + c8 + b;
        cur[b] = (i0 < mp && c < nct) ? *reinterpret_cast<const V4 *>(F + (k + i0) + (k + ncols + coff + c) * ld)
                                      : v4_zero<T>();
    }
    for (int idx = threadIdx.x; idx < NB * (TC_ROWS / 4); idx += 256) {
        const int ll = idx / (TC_ROWS / 4), q = idx % (TC_ROWS / 4);
        const int64_t i = rbase + 4 * q;
        *reinterpret_cast<V4 *>(&sV[ll][4 * q]) = (i < mp) ? v_quad(F, ld, k, i, ll, ncols) : v4_zero<T>();
    }
    for (int idx = threadIdx.x; idx < NB * TC_COLS; idx += 256) {
        const int ll = idx / TC_COLS, cc = idx % TC_COLS;
        const int64_t c = cbase + cc;
        sZ[ll][cc] = (c < nct) ? Z[(int64_t)ll * nct + c] : T(0);
    }
    __syncthreads();
    T acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = T(0);
#pragma unroll 4
    for (int ll = 0; ll < NB; ++ll) {
        const V4 v = *reinterpret_cast<const V4 *>(&sV[ll][r4]);
        const V4 z0 = *reinterpret_cast<const V4 *>(&sZ[ll][c8]);
        const V4 z1 = *reinterpret_cast<const V4 *>(&sZ[ll][c8 + 4]);
        const T zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            acc[0][b] += v.x * zz[b];
            acc[1][b] += v.y * zz[b];
            acc[2][b] += v.z * zz[b];
            acc[3][b] += v.w * zz[b];
        }
    }
    if (i0 >= mp) return;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int64_t c = cbase + c8 + b;
        if (c >= nct) break;
        V4 u = cur[b];
        u.x -= acc[0][b];
        u.y -= acc[1][b];
        u.z -= acc[2][b];
        u.w -= acc[3][b];
        *reinterpret_cast<V4 *>(F + (k + i0) + (k + ncols + coff + c) * ld) = u;
    }
}

// Sum of vals[0..NB) over the 32 lanes, scattered: on exit lane L holds the sum for
// index L % NB in vals[0] (butterfly for the lane bits above NB, then a
// reduce-scatter with NB - 1 shuffles).
template <typename T, int NB>
__device__ __forceinline__ T warp_reduce_scatter(T (&vals)[NB], int lane)
{
#pragma unroll
    for (int s = 16; s >= NB; s >>= 1)
#pragma unroll
        for (int i = 0; i < NB; ++i) vals[i] += __shfl_xor_sync(0xffffffffu, vals[i], s);
#pragma unroll
    for (int s = NB / 2; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            T send = up ? vals[i] : vals[i + s];
            T keep = up ? vals[i + s] : vals[i];
            vals[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return vals[0];
}

// y <- Q^T y (transpose) or Q y for a vector y [m_aug] of type T, grid-wide: one
// CTA per SM (cooperative launch) owns a contiguous chunk of rows.  Per panel p:
// dots s_l = sum_i V(i,l) y_i (CTA partials, double-buffered in global memory,
// one grid barrier), w = T^T s (Q^T) or T s (Q), then y_i -= sum_l V(i,l) w_l on
// the owned rows.  Rows below the unit-diagonal block read V without masking.
constexpr int AQ_THREADS = 256;

template <typename T, int NB>
__global__ void __launch_bounds__(AQ_THREADS, 1)
k_apply_q_grid(const T *__restrict__ F, int64_t ld, int64_t m_aug, int64_t n,
               const T *__restrict__ Tall, T *__restrict__ y, int transpose, T *__restrict__ part,
               GridBar *bar, int *flag)
{
    constexpr int NW = AQ_THREADS / 32;
    constexpr int GROUPS = AQ_THREADS / NB;
    __shared__ T red[NW][NB];
    __shared__ T red2[GROUPS][NB];
    __shared__ T w[NB];
    __shared__ T sT[NB][NB + 1];
    __shared__ volatile int s_abort;
    const unsigned G = gridDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_abort = 0;
    const int64_t rows_per = fl_cdiv_dev(m_aug, G);
    const int64_t r_lo = (int64_t)blockIdx.x * rows_per, r_hi = fl_min64(m_aug, r_lo + rows_per);
    const int npanels = (int)((n + NB - 1) / NB);
    for (int step = 0; step < npanels; ++step) {
        const int p = transpose ? step : (npanels - 1 - step);
        const int64_t k = (int64_t)p * NB;
        const int ncols = (int)fl_min64(NB, n - k);
        const int par = step & 1;
        const T *Vp = F + k + k * ld;
        T acc[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) acc[q] = T(0);
        for (int64_t i = fl_max64(r_lo, k) + threadIdx.x; i < r_hi; i += AQ_THREADS) {
            const int64_t li = i - k;
            const T yi = y[i];
            if (li >= NB) {
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (q < ncols) acc[q] += Vp[li + q * ld] * yi;
            } else {
#pragma unroll
                for (int q = 0; q < NB; ++q) acc[q] += v_at(F, ld, k, li, q, ncols) * yi;
            }
        }
        const T partial = warp_reduce_scatter<T, NB>(acc, lane);
        if (lane < NB) red[warp][lane] = partial;
        __syncthreads();
        if (warp == 0 && lane < NB) {
            T s = T(0);
#pragma unroll
            for (int ww = 0; ww < NW; ++ww) s += red[ww][lane];
            part[((int64_t)par * G + blockIdx.x) * NB + lane] = s;
        }
        if (!grid_sync(bar, G, flag, &s_abort)) return;
        for (int idx = threadIdx.x; idx < NB * NB; idx += AQ_THREADS)
            sT[idx % NB][idx / NB] = Tall[(int64_t)p * NB * NB + idx];
        {   // sum the G partials: thread (group g, column l) takes CTAs g, g + GROUPS, ...
            const int l = threadIdx.x % NB, g = threadIdx.x / NB;
            T s0 = T(0), s1 = T(0);
            unsigned c = g;
            for (; c + GROUPS < G; c += 2 * GROUPS) {
                s0 += part[((int64_t)par * G + c) * NB + l];
                s1 += part[((int64_t)par * G + c + GROUPS) * NB + l];
            }
            for (; c < G; c += GROUPS) s0 += part[((int64_t)par * G + c) * NB + l];
            red2[g][l] = s0 + s1;
        }
        __syncthreads();
        if (warp == 0) {
            T s = T(0);
            if (lane < NB)
#pragma unroll
                for (int g = 0; g < GROUPS; ++g) s += red2[g][lane];
            T wl = T(0);
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const T sq = __shfl_sync(0xffffffffu, s, q);
                if (lane < NB) {
                    // Q^T: w = T^T s -> w_l = sum_{q <= l} T(q,l) s_q ; Q: w = T s -> w_l = sum_{q >= l} T(l,q) s_q
                    if (transpose) { if (q <= lane) wl += sT[q][lane] * sq; }
                    else { if (q >= lane) wl += sT[lane][q] * sq; }
                }
            }
            if (lane < NB) w[lane] = wl;
        }
        __syncthreads();
        for (int64_t i = fl_max64(r_lo, k) + threadIdx.x; i < r_hi; i += AQ_THREADS) {
            const int64_t li = i - k;
            T s = T(0);
            if (li >= NB) {
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    if (q < ncols) s += Vp[li + q * ld] * w[q];
            } else {
#pragma unroll
                for (int q = 0; q < NB; ++q) s += v_at(F, ld, k, li, q, ncols) * w[q];
            }
            y[i] -= s;
        }
        __syncthreads();
    }
}

// Copy A (and the rhs columns) into the factor storage, writing the Tikhonov
// rows sqrt(mu) I below the m real rows when mu > 0.
template <typename TA, typename T>
__global__ void k_copy_in(const TA *__restrict__ A, int64_t ldA, int64_t m, int64_t n,
                          double sqrt_mu, int64_t m_aug, const double *__restrict__ rhs,
                          int64_t ld_rhs, int nrhs, T *__restrict__ F, int64_t ld)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = blockIdx.y;
    if (i >= ld) return;
    T v;
    if (i >= m_aug) v = T(0);          // padding rows stay zero through the factorisation
    else if (c < n) v = (i < m) ? (T)A[i + c * ldA] : ((i - m == c) ? (T)sqrt_mu : T(0));
    else v = (i < m) ? (T)rhs[i + (c - n) * ld_rhs] : T(0);
    F[i + c * ld] = v;
}

// Residual of the augmented system in FP64:  r_i = rhs_i - sum_j A_ij beta_j
// (i < m), r_{m+j} = -sqrt(mu) beta_j.  Column-split partial sums, fixed-order
// reduction; the second kernel also rounds r to the factor type for the
// correction solve and accumulates ||r||^2 per block.
constexpr int RES_ROWS = 256;
constexpr int RES_COLS = 128;

__global__ void __launch_bounds__(RES_ROWS)
k_resid_partial(const double *__restrict__ A, int64_t ldA, int64_t m, int64_t n,
                const double *__restrict__ beta, double *__restrict__ part)
{
    __shared__ double sb[RES_COLS];
    const int64_t j0 = (int64_t)blockIdx.y * RES_COLS;
    const int nc = (int)fl_min64(RES_COLS, n - j0);
    for (int t = threadIdx.x; t < nc; t += blockDim.x) sb[t] = beta[j0 + t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * RES_ROWS + threadIdx.x;
    if (i >= m) return;
    double acc = 0.0;
    const double *a = A + i + j0 * ldA;
#pragma unroll 8
    for (int c = 0; c < nc; ++c) acc = fma(a[(int64_t)c * ldA], sb[c], acc);
    part[(int64_t)blockIdx.y * m + i] = acc;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_resid_finish(const double *__restrict__ part, int nsplit, const double *__restrict__ rhs,
               const double *__restrict__ beta, int64_t m, int64_t n, double sqrt_mu,
               int64_t m_aug, T *__restrict__ r_out, double *__restrict__ norm_part)
{
    __shared__ double red[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double r = 0.0;
    if (i < m) {
        double s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += part[(int64_t)sp * m + i];
        r = rhs[i] - s;
    } else if (i < m_aug) {
        r = -sqrt_mu * beta[i - m];
    }
    if (i < m_aug) r_out[i] = (T)r;
    red[threadIdx.x] = r * r;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) norm_part[blockIdx.x] = red[0];
}

template <typename T>
__global__ void k_extract_rhs(const T *__restrict__ F, int64_t ld, int64_t n, int r,
                              T *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = F[i + (n + r) * ld];
}

template <typename T>
__global__ void k_to_f64(const T *__restrict__ src, int64_t n, double *__restrict__ dst, int add,
                         const int *skip)
{
    if (skip && *skip) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (add) dst[i] += (double)src[i];
    else dst[i] = (double)src[i];
}

template <typename T>
__global__ void k_from_f64(const double *__restrict__ src, int64_t n, int64_t n_total,
                           T *__restrict__ dst, const int *skip)
{
    if (skip && *skip) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_total) dst[i] = (i < n) ? (T)src[i] : T(0);
}

__global__ void k_sum_norm(const double *__restrict__ part, int n, double *__restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = sqrt(s);
    }
}

// Allow the largest dynamic shared memory the kernel can take next to its static part.
template <typename K>
cudaError_t set_max_dynamic_smem(K kernel, int optin)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                optin - (int)a.sharedSizeBytes);
}

template <typename T, int NB>
int set_panel_attrs(fastlsq_ctx *ctx)
{
    static FlOncePerDevice once;
    if (!once.pending(ctx->device)) return 0;
    cudaError_t e = set_max_dynamic_smem(k_panel<T, NB>, ctx->max_smem_optin);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_panel<T, NB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);

    if (e != cudaSuccess) return fl_cuda(ctx, e, "cudaFuncSetAttribute");
    once.done(ctx->device);
    return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

int fl_panel_capacity_nb(fastlsq_ctx *ctx, int64_t m_aug, size_t elem)
{
    // largest NB in {32, 16, 8} whose panel slice fits on a 16-CTA cluster
    for (int nb = 32; nb >= 8; nb /= 2) {
        int64_t rpc = fl_cdiv(m_aug, CL_MAX);
        size_t bytes = elem * ((size_t)rpc * (nb + 1) + PANEL_WARPS * 33 + 2 * (CL_MAX + 1) * nb +
                               2 * nb * (nb + 1) + nb);
        if (bytes <= (size_t)ctx->max_smem_optin) return nb;
    }
    return 0;
}

template <typename T, int NB>
static int launch_panel(fastlsq_ctx *ctx, T *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                        T *tau, T *Tblk)
{
    FL_TRY((set_panel_attrs<T, NB>(ctx)));
    const int64_t mp = m_aug - k;
    int CL = CL_MAX;
    while (CL > 1 && fl_cdiv(mp, CL) < NB) CL >>= 1;
    int rpc = (int)fl_cdiv(mp, CL);
    if (rpc < ncols) rpc = ncols;
    size_t smem = PanelSmem<T, NB>::bytes(rpc);
    if (smem > (size_t)ctx->max_smem_optin)
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "panel of %lld rows exceeds the on-chip capacity",
                       (long long)mp);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(PANEL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    FL_PROF(ctx, FASTLSQ_K_PANEL);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_panel<T, NB>, F, ld, k, m_aug, ncols, rpc, tau, Tblk,
                                       ctx->d_flag);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "panel launch");
    return 0;
}

template <typename T, int NB, bool TFWD = false>
static int launch_trailing(fastlsq_ctx *ctx, T *F, int64_t ld, int64_t k, int64_t m_aug,
                           int ncols, int64_t nct, int64_t coff, const T *Tblk, int *counters)
{
    if (nct <= 0) return 0;
    const int64_t mp = m_aug - k;
    const int64_t ctiles = fl_cdiv(nct, TY_COLS);
    // split the long row dimension so the grid covers the GPU about twice, with at least
    // ctx->split_rows rows per split (256 by default: the shortest latency of one narrow
    // update inside an outer block at 36,864 rows; larger splits use fewer CTAs)
    int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>(fl_cdiv(2 * ctx->num_sms, ctiles),
                                                            fl_cdiv(mp, ctx->split_rows)));
    nsplit = std::min<int64_t>(nsplit, TREE_MAX_SPLITS);
    int64_t rows_per_split = fl_round_up(fl_cdiv(mp, nsplit), TY_ROWS);
    nsplit = fl_cdiv(mp, rows_per_split);
    T *Ypart = (T *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(T) * nsplit * NB * nct);
    T *Z = (T *)fl_ws(ctx, FL_WS_ZBUF, sizeof(T) * NB * nct);
    if (!Ypart || !Z) return FASTLSQ_ERR_NOMEM;
    static FlOncePerDevice attr_once;
    const size_t smem_c = sizeof(T) * NB * (TC_COLS + TC_ROWS);
    if (attr_once.pending(ctx->device)) {
        cudaError_t e = cudaFuncSetAttribute(k_trail_c<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_c);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_trail_y<T, NB, TFWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)TrailYSmem<T, NB>::bytes);
        if (e != cudaSuccess) return fl_cuda(ctx, e, "trailing-update attributes");
        attr_once.done(ctx->device);
    }
    FL_PROF_N(ctx, FASTLSQ_K_TRAIL_SIMT, 2);
    k_trail_y<T, NB, TFWD><<<dim3((unsigned)ctiles, (unsigned)nsplit), TY_THREADS, TrailYSmem<T, NB>::bytes,
                             ctx->stream>>>(F, ld, k, m_aug, ncols, nct, coff, rows_per_split, Ypart, Z, Tblk, counters);
    FL_CHECK_LAUNCH(ctx, "trail_y");
    k_trail_c<T, NB><<<dim3((unsigned)fl_cdiv(mp, TC_ROWS), (unsigned)fl_cdiv(nct, TC_COLS)), 256, smem_c,
                       ctx->stream>>>(F, ld, k, m_aug, ncols, nct, coff, Z);
    FL_CHECK_LAUNCH(ctx, "trail_c");
    return 0;
}

template <typename T, int NB>
static int panel_any(fastlsq_ctx *ctx, T *F, int64_t ld, int64_t k, int64_t m_aug, int ncols, T *tau,
                     T *Tblk)
{
    if constexpr (std::is_same<T, float>::value && NB == 32) {
        if (ctx->panel_reg && fl_panel_reg_fits(m_aug - k))
            return fl_panel_reg_f32(ctx, F, ld, k, m_aug, ncols, tau, Tblk);
    }
    if constexpr (std::is_same<T, float>::value && NB == 16) {
        if (ctx->panel_reg && fl_panel_tall_fits(ctx, m_aug - k, false))
            return fl_panel_tall_f32(ctx, F, ld, k, m_aug, ncols, tau, Tblk);
    }
    return launch_panel<T, NB>(ctx, F, ld, k, m_aug, ncols, tau, Tblk);
}

// trailing columns [k + ncols + coff, k + ncols + coff + nct) updated by panel k
template <typename T, int NB>
static int trailing_any(fastlsq_ctx *ctx, T *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                        int64_t nct, int64_t coff, int64_t ntot, const T *Tblk, int *counters, int use_tc)
{
    if (nct <= 0) return 0;
    if constexpr (std::is_same<T, float>::value) {
        if (use_tc) {
            const int rc = fl_trailing_tc_f32(ctx, F, ld, k, m_aug, ncols, NB, nct, coff, ntot, Tblk, counters);
            if (rc != 1) return rc;
        }
    }
    return launch_trailing<T, NB>(ctx, F, ld, k, m_aug, ncols, nct, coff, Tblk, counters);
}

// Blocked right-looking Householder QR.  With look-ahead, panel p's update of the
// next panel's columns runs first; the rest of panel p's update is then handed to
// the auxiliary stream while the next panel is factored right away on the caller's
// stream (so the panel's cluster is placed before the update's CTAs fill the GPU),
// and the two join before panel p+1's own update.
template <typename T, int NB>
static int factor_t(fastlsq_ctx *ctx, T *F, int64_t ld, int64_t m_aug, int64_t n, int nrhs,
                    T *tau, T *Tall, int use_tc)
{
    const int64_t ntot = n + nrhs;
    // one completion counter per column tile of the trailing updates, zero between panels
    const int64_t max_tiles = fl_cdiv(ntot, 32) + 8;
    const size_t cbytes = sizeof(int) * (size_t)max_tiles * TREE_STRIDE;
    int *counters = (int *)fl_ws(ctx, FL_WS_COUNTERS, cbytes);
    if (!counters) return FASTLSQ_ERR_NOMEM;
    cudaMemsetAsync(counters, 0, cbytes, ctx->stream);
    const int64_t npan = fl_cdiv(n, NB);
    const bool la = ctx->lookahead && ctx->aux_stream && npan > 1;
    for (int64_t p = 0; p < npan; ++p) {
        const int64_t k = p * NB;
        const int ncols = (int)std::min<int64_t>(NB, n - k);
        T *Tblk = Tall + p * NB * NB;
        if (!la || p == 0) FL_TRY((panel_any<T, NB>(ctx, F, ld, k, m_aug, ncols, tau + k, Tblk)));
        const int64_t nct = ntot - (k + ncols);
        if (la && p + 1 < npan) {
            const int ncn = (int)std::min<int64_t>(NB, n - (k + NB));
            // the next panel can take panel p's update of its own columns in its prologue
            bool fuse = false;
            if constexpr (std::is_same<T, float>::value && NB == 32)
                fuse = ctx->panel_reg && ctx->fuse_next && fl_panel_reg_fits(m_aug - (k + NB)) &&
                       fl_panel_reg_fused_fits(ctx, m_aug - (k + NB));
            if (!fuse)
                FL_TRY((trailing_any<T, NB>(ctx, F, ld, k, m_aug, ncols, ncn, 0, ntot, Tblk, counters, use_tc)));
            cudaError_t e = cudaEventRecord(ctx->ev_fork, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_fork, 0);
            if (e != cudaSuccess) return fl_cuda(ctx, e, "look-ahead fork");
            cudaStream_t main_stream = ctx->stream;
            ctx->stream = ctx->aux_stream;
            const int rc = trailing_any<T, NB>(ctx, F, ld, k, m_aug, ncols, nct - ncn, ncn, ntot, Tblk, counters,
                                               use_tc);
            if (rc == 0) e = cudaEventRecord(ctx->ev_join, ctx->aux_stream);
            ctx->stream = main_stream;
            FL_TRY(rc);
            if (e != cudaSuccess) return fl_cuda(ctx, e, "look-ahead join");
            if (fuse) {
                if constexpr (std::is_same<T, float>::value && NB == 32)
                    FL_TRY(fl_panel_reg_f32(ctx, F, ld, k + NB, m_aug, ncn, tau + k + NB, Tblk + NB * NB, k, Tblk));
            } else {
                FL_TRY((panel_any<T, NB>(ctx, F, ld, k + NB, m_aug, ncn, tau + k + NB, Tblk + NB * NB)));
            }
            e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
            if (e != cudaSuccess) return fl_cuda(ctx, e, "look-ahead join");
        } else {
            FL_TRY((trailing_any<T, NB>(ctx, F, ld, k, m_aug, ncols, nct, 0, ntot, Tblk, counters, use_tc)));
        }
    }
    return 0;
}

// Two-level blocked Householder QR of an FP32 factor: outer blocks of 128 columns,
// each factored as inner panels of width NB (panel kernel, then the SIMT update of the
// block's remaining columns, K = NB); the block's reflectors then update every column
// right of the block at once on the tensor cores (fl_block_update_f32: K = 128, three-part
// bf16 split).  The factor's storage (reflectors, tau, per-panel T) is the same as the
// one-level schedule's, so every solve reads it unchanged.
template <int NB>
static int factor_blocked(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t m_aug, int64_t n, int nrhs,
                          float *tau, float *Tall, float *Tball, int *tb_ok)
{
    constexpr int BLK = 128;
    if (tb_ok) *tb_ok = 0;
    float *Gall = nullptr;
    if (Tball) {
        Gall = (float *)fl_ws(ctx, FL_WS_BLK_G, sizeof(float) * (size_t)fl_cdiv(n, BLK) * BLK * BLK);
        if (!Gall) return FASTLSQ_ERR_NOMEM;
    }
    bool all_g = Gall != nullptr;
    const int64_t ntot = n + nrhs;
    const int64_t max_tiles = fl_cdiv(ntot, 32) + 8;
    const size_t cbytes = sizeof(int) * (size_t)max_tiles * TREE_STRIDE;
    int *counters = (int *)fl_ws(ctx, FL_WS_COUNTERS, cbytes);
    if (!counters) return FASTLSQ_ERR_NOMEM;
    cudaMemsetAsync(counters, 0, cbytes, ctx->stream);
    const bool la = ctx->lookahead && ctx->aux_stream && ctx->panel_reg && ctx->fuse_next;
    const int split = (ctx->lookahead && ctx->aux2_stream) ? 1 : 0;
    for (int64_t k = 0; k < n; k += BLK) {
        const int nbk = (int)std::min<int64_t>(BLK, n - k);
        bool factored = false;        // this inner panel was factored by the previous step's look-ahead
        for (int64_t kp = k; kp < k + nbk; kp += NB) {
            const int ncols = (int)std::min<int64_t>(NB, n - kp);
            float *Tblk = Tall + (kp / NB) * NB * NB;
            if (!factored) FL_TRY((panel_any<float, NB>(ctx, F, ld, kp, m_aug, ncols, tau + kp, Tblk)));
            factored = false;
            const int64_t nin = k + nbk - (kp + ncols);
            if (nin <= 0) continue;
            // look-ahead (tall 16-wide panels): the next panel applies this panel's update
            // to its own columns in its prologue, and the rest of the update runs on the
            // auxiliary stream beside it; the two join before the panel after next
            bool fuse = false;
            if constexpr (NB == 16) fuse = la && fl_panel_tall_fits(ctx, m_aug - (kp + NB), true);
            if (!fuse) {
                FL_TRY((launch_trailing<float, NB>(ctx, F, ld, kp, m_aug, ncols, nin, 0, Tblk, counters)));
                continue;
            }
            const int ncn = (int)std::min<int64_t>(NB, nin);
            const bool rest = nin > ncn;
            if (rest) {
                cudaError_t e = cudaEventRecord(ctx->ev_fork, ctx->stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_fork, 0);
                if (e != cudaSuccess) return fl_cuda(ctx, e, "look-ahead fork");
            }
            // the panel is submitted first (and its stream has the higher priority), so
            // that its cluster is placed before the update's CTAs fill the GPU
            FL_TRY(fl_panel_tall_f32(ctx, F, ld, kp + NB, m_aug, ncn, tau + kp + NB, Tblk + NB * NB, kp, Tblk));
            if (rest) {
                cudaStream_t main_stream = ctx->stream;
                ctx->stream = ctx->aux_stream;
                const int rc = launch_trailing<float, NB>(ctx, F, ld, kp, m_aug, ncols, nin - ncn, ncn, Tblk,
                                                          counters);
                cudaError_t e = cudaSuccess;
                if (rc == 0) e = cudaEventRecord(ctx->ev_join, ctx->aux_stream);
                ctx->stream = main_stream;
                FL_TRY(rc);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0);
                if (e != cudaSuccess) return fl_cuda(ctx, e, "look-ahead join");
            }
            factored = true;
        }
        if (ntot <= k + nbk) {
            all_g = false;
            continue;
        }
        // with look-ahead, the next block's columns are updated first and its panels start
        // while the rest of this block's update pass runs beside them
        const int rc = fl_block_update_f32(ctx, F, ld, k, m_aug, nbk, ntot, NB, Tall + (k / NB) * NB * NB,
                                           Gall ? Gall + (k / BLK) * BLK * BLK : nullptr, split);
        if (rc < 0) {
            fl_block_join(ctx);
            return rc;
        }
        if (rc == 1) {      // shape not taken: the block's panels update the columns one by one
            all_g = false;
            for (int64_t kp = k; kp < k + nbk; kp += NB) {
                const int ncols = (int)std::min<int64_t>(NB, n - kp);
                FL_TRY((launch_trailing<float, NB>(ctx, F, ld, kp, m_aug, ncols, ntot - (k + nbk),
                                                   (k + nbk) - (kp + ncols), Tall + (kp / NB) * NB * NB,
                                                   counters)));
            }
        }
    }
    FL_TRY(fl_block_join(ctx));
    if (all_g) {
        FL_TRY(fl_block_t_f32(ctx, Gall, Tall, n, NB, Tball));
        if (tb_ok) *tb_ok = 1;
    }
    return 0;
}

template <typename T>
int fl_factor(fastlsq_ctx *ctx, T *F, int64_t ld, int64_t m_aug, int64_t n, int nrhs, int nb,
              T *tau, T *Tall, int use_tc, float *Tball, int *tb_ok)
{
    if (tb_ok) *tb_ok = 0;
    if constexpr (std::is_same<T, float>::value) {
        if (use_tc == FL_TC_BLOCKED) {
            if (nb == 32) return factor_blocked<32>(ctx, F, ld, m_aug, n, nrhs, tau, Tall, Tball, tb_ok);
            if (nb == 16) return factor_blocked<16>(ctx, F, ld, m_aug, n, nrhs, tau, Tall, Tball, tb_ok);
        }
    }
    switch (nb) {
    case 32: return factor_t<T, 32>(ctx, F, ld, m_aug, n, nrhs, tau, Tall, use_tc);
    case 16: return factor_t<T, 16>(ctx, F, ld, m_aug, n, nrhs, tau, Tall, use_tc);
    case 8: return factor_t<T, 8>(ctx, F, ld, m_aug, n, nrhs, tau, Tall, use_tc);
    default: return fl_fail(ctx, FASTLSQ_ERR_INVALID, "panel width %d", nb);
    }
}
template int fl_factor<float>(fastlsq_ctx *, float *, int64_t, int64_t, int64_t, int, int, float *,
                              float *, int, float *, int *);
template int fl_factor<double>(fastlsq_ctx *, double *, int64_t, int64_t, int64_t, int, int,
                               double *, double *, int, float *, int *);

template <typename T>
int fl_apply_q(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t m_aug, int64_t n, int nb,
               const T *Tall, T *y, int transpose, const float *Tball)
{
    if constexpr (std::is_same<T, float>::value) {
        if (Tball) {
            const int rc = fl_apply_qb_f32(ctx, F, ld, m_aug, n, Tball, y, transpose);
            if (rc <= 0) return rc;      // 1: shape not taken by the block-reflector kernel
        }
        const int rc = fl_apply_q_cluster<float>(ctx, F, ld, m_aug, n, nb, Tall, y, transpose);
        if (rc <= 0) return rc;          // 1: shape not taken by the cluster kernel
    }
    // about 512 rows per CTA keeps the partial sums few (one L2 round trip to combine)
    const unsigned G = (unsigned)std::min<int64_t>(ctx->num_sms, std::max<int64_t>(4, fl_cdiv(m_aug, 512)));
    T *part = (T *)fl_ws(ctx, FL_WS_APPLYQ, sizeof(T) * 2 * ctx->num_sms * 32);
    if (!part) return FASTLSQ_ERR_NOMEM;
    GridBar *bar = (GridBar *)ctx->d_grid_bar;
    int *flag = ctx->d_flag;
    void *args[] = {(void *)&F, (void *)&ld, (void *)&m_aug, (void *)&n, (void *)&Tall, (void *)&y,
                    (void *)&transpose, (void *)&part, (void *)&bar, (void *)&flag};
    const void *fn = nullptr;
    switch (nb) {
    case 32: fn = (const void *)k_apply_q_grid<T, 32>; break;
    case 16: fn = (const void *)k_apply_q_grid<T, 16>; break;
    case 8: fn = (const void *)k_apply_q_grid<T, 8>; break;
    default: return fl_fail(ctx, FASTLSQ_ERR_INVALID, "panel width %d", nb);
    }
    FL_PROF(ctx, FASTLSQ_K_APPLY_Q);
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(AQ_THREADS), args, 0, ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "apply_q launch");
    return 0;
}
template int fl_apply_q<float>(fastlsq_ctx *, const float *, int64_t, int64_t, int64_t, int,
                               const float *, float *, int, const float *);
template int fl_apply_q<double>(fastlsq_ctx *, const double *, int64_t, int64_t, int64_t, int,
                                const double *, double *, int, const float *);

// E = [I_n; 0] (ld rows, the padding rows included, n columns)
__global__ void k_eye(double *__restrict__ E, int64_t ld, int64_t n)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ld * n) return;
    const int64_t i = idx % ld, j = idx / ld;
    E[idx] = (i == j) ? 1.0 : 0.0;
}

// The thin Q of an FP64 factor: columns [col0, col0 + n) of F (which holds the factor
// in its first n columns, leading dimension ld) become Q [I_n; 0] = H_0 H_1 ... H_{P-1}
// [I_n; 0].  The panels are applied last to first by the SIMT narrow update with Z = T Y
// (each H_p = I - V_p T_p V_p^T); panel p touches rows [k_p, m_aug) and only the
// columns [k_p, n) of E, since E's columns left of k_p are still unit vectors above
// row k_p there (as in LAPACK's orgqr).  About m n^2 - n^3 / 3 FMAs, the work of the
// factorisation's own updates.
template <int NB>
static int form_q_nb(fastlsq_ctx *ctx, double *F, int64_t ld, int64_t m_aug, int64_t n, const double *Tall,
                     int64_t col0)
{
    const int64_t max_tiles = fl_cdiv(n, 32) + 8;
    const size_t cbytes = sizeof(int) * (size_t)max_tiles * TREE_STRIDE;
    int *counters = (int *)fl_ws(ctx, FL_WS_COUNTERS, cbytes);
    if (!counters) return FASTLSQ_ERR_NOMEM;
    cudaError_t e = cudaMemsetAsync(counters, 0, cbytes, ctx->stream);
    if (e != cudaSuccess) return fl_cuda(ctx, e, "form_q counters");
    k_eye<<<(unsigned)fl_cdiv(ld * n, 256), 256, 0, ctx->stream>>>(F + col0 * ld, ld, n);
    FL_CHECK_LAUNCH(ctx, "form_q eye");
    const int64_t npan = fl_cdiv(n, NB);
    for (int64_t p = npan - 1; p >= 0; --p) {
        const int64_t k = p * NB;
        const int ncols = (int)std::min<int64_t>(NB, n - k);
        FL_TRY((launch_trailing<double, NB, true>(ctx, F, ld, k, m_aug, ncols, n - k, col0 - ncols,
                                                  Tall + p * NB * NB, counters)));
    }
    return 0;
}

int fl_form_q_f64(fastlsq_ctx *ctx, double *F, int64_t ld, int64_t m_aug, int64_t n, int nb, const double *Tall,
                  int64_t col0)
{
    if (col0 < n || m_aug < n || ld < m_aug || (ld & 3))
        return fl_fail(ctx, FASTLSQ_ERR_INVALID, "form_q: shape");
    switch (nb) {
    case 32: return form_q_nb<32>(ctx, F, ld, m_aug, n, Tall, col0);
    case 16: return form_q_nb<16>(ctx, F, ld, m_aug, n, Tall, col0);
    case 8: return form_q_nb<8>(ctx, F, ld, m_aug, n, Tall, col0);
    default: return fl_fail(ctx, FASTLSQ_ERR_INVALID, "panel width %d", nb);
    }
}

template <typename TA, typename T>
int fl_copy_in(fastlsq_ctx *ctx, const TA *A, int64_t ldA, int64_t m, int64_t n, double mu,
               int64_t m_aug, const double *rhs, int64_t ld_rhs, int nrhs, T *F, int64_t ld)
{
    dim3 grid((unsigned)fl_cdiv(ld, 256), (unsigned)(n + nrhs));
    FL_PROF(ctx, FASTLSQ_K_COPY_IN);
    k_copy_in<TA, T><<<grid, 256, 0, ctx->stream>>>(A, ldA, m, n, mu > 0 ? sqrt(mu) : 0.0, m_aug,
                                                    rhs, ld_rhs, nrhs, F, ld);
    FL_CHECK_LAUNCH(ctx, "copy_in");
    return 0;
}
template int fl_copy_in<float, float>(fastlsq_ctx *, const float *, int64_t, int64_t, int64_t,
                                      double, int64_t, const double *, int64_t, int, float *,
                                      int64_t);
template int fl_copy_in<double, float>(fastlsq_ctx *, const double *, int64_t, int64_t, int64_t,
                                       double, int64_t, const double *, int64_t, int, float *,
                                       int64_t);
template int fl_copy_in<double, double>(fastlsq_ctx *, const double *, int64_t, int64_t, int64_t,
                                        double, int64_t, const double *, int64_t, int, double *,
                                        int64_t);

template <typename T>
int fl_residual(fastlsq_ctx *ctx, const double *A, int64_t ldA, int64_t m, int64_t n, double mu,
                int64_t m_aug, const double *rhs, const double *beta, T *r_out, double *norm_out)
{
    int nsplit = (int)fl_cdiv(n, RES_COLS);
    double *part = (double *)fl_ws(ctx, FL_WS_PARTIAL, sizeof(double) * nsplit * m);
    int nblk = (int)fl_cdiv(m_aug, 256);
    double *npart = (double *)fl_ws(ctx, FL_WS_SCALARS, sizeof(double) * (nblk + 8));
    if (!part || !npart) return FASTLSQ_ERR_NOMEM;
    FL_PROF_N(ctx, FASTLSQ_K_RESIDUAL, norm_out ? 3 : 2);
    k_resid_partial<<<dim3((unsigned)fl_cdiv(m, RES_ROWS), (unsigned)nsplit), RES_ROWS, 0,
                      ctx->stream>>>(A, ldA, m, n, beta, part);
    FL_CHECK_LAUNCH(ctx, "resid_partial");
    k_resid_finish<T><<<nblk, 256, 0, ctx->stream>>>(part, nsplit, rhs, beta, m, n,
                                                     mu > 0 ? sqrt(mu) : 0.0, m_aug, r_out, npart);
    FL_CHECK_LAUNCH(ctx, "resid_finish");
    if (norm_out) {
        k_sum_norm<<<1, 32, 0, ctx->stream>>>(npart, nblk, norm_out);
        FL_CHECK_LAUNCH(ctx, "sum_norm");
    }
    return 0;
}
template int fl_residual<float>(fastlsq_ctx *, const double *, int64_t, int64_t, int64_t, double,
                                int64_t, const double *, const double *, float *, double *);
template int fl_residual<double>(fastlsq_ctx *, const double *, int64_t, int64_t, int64_t, double,
                                 int64_t, const double *, const double *, double *, double *);

template <typename T>
int fl_extract_rhs(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t n, int r, T *out)
{
    FL_PROF(ctx, FASTLSQ_K_VECTOR);
    k_extract_rhs<T><<<(unsigned)fl_cdiv(n, 256), 256, 0, ctx->stream>>>(F, ld, n, r, out);
    FL_CHECK_LAUNCH(ctx, "extract_rhs");
    return 0;
}
template int fl_extract_rhs<float>(fastlsq_ctx *, const float *, int64_t, int64_t, int, float *);
template int fl_extract_rhs<double>(fastlsq_ctx *, const double *, int64_t, int64_t, int, double *);

template <typename T>
int fl_to_f64(fastlsq_ctx *ctx, const T *src, int64_t n, double *dst, int add, const int *skip)
{
    FL_PROF(ctx, FASTLSQ_K_VECTOR);
    k_to_f64<T><<<(unsigned)fl_cdiv(n, 256), 256, 0, ctx->stream>>>(src, n, dst, add, skip);
    FL_CHECK_LAUNCH(ctx, "to_f64");
    return 0;
}
template int fl_to_f64<float>(fastlsq_ctx *, const float *, int64_t, double *, int, const int *);
template int fl_to_f64<double>(fastlsq_ctx *, const double *, int64_t, double *, int, const int *);

template <typename T>
int fl_from_f64(fastlsq_ctx *ctx, const double *src, int64_t n, int64_t n_total, T *dst,
                const int *skip)
{
    FL_PROF(ctx, FASTLSQ_K_VECTOR);
    k_from_f64<T><<<(unsigned)fl_cdiv(n_total, 256), 256, 0, ctx->stream>>>(src, n, n_total, dst, skip);
    FL_CHECK_LAUNCH(ctx, "from_f64");
    return 0;
}
template int fl_from_f64<float>(fastlsq_ctx *, const double *, int64_t, int64_t, float *,
                                const int *);
template int fl_from_f64<double>(fastlsq_ctx *, const double *, int64_t, int64_t, double *,
                                 const int *);

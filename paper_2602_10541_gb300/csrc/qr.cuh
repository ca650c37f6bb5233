// Launchers of the blocked Householder QR and its solves (qr.cu, tc_update.cu).
#pragma once
#include <cuda.h>

#include "common.cuh"

__host__ __device__ __forceinline__ int64_t fl_cdiv_dev(int64_t a, int64_t b) { return (a + b - 1) / b; }

int fl_panel_capacity_nb(fastlsq_ctx *ctx, int64_t m_aug, size_t elem);

// Tball (two-level FP32 factor, may be null): receives every outer block's T_b; *tb_ok
// tells whether all of them were formed (a block whose update was not taken has none)
template <typename T>
int fl_factor(fastlsq_ctx *ctx, T *F, int64_t ld, int64_t m_aug, int64_t n, int nrhs, int nb,
              T *tau, T *Tall, int use_tc, float *Tball = nullptr, int *tb_ok = nullptr);
// Q^T y / Q y on one cluster, FP32 factor with panel width 32 (apply_q.cu); returns 1
// when the shape is not taken (more than 16 x 640 rows or another panel width)
template <typename T>
int fl_apply_q_cluster(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t m_aug, int64_t n, int nb,
                       const T *Tall, T *y, int transpose);
// Tball: the two-level factor's block reflectors' T (or null): then one grid barrier
// per outer block (apply_qb.cu) where the shape fits
template <typename T>
int fl_apply_q(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t m_aug, int64_t n, int nb,
               const T *Tall, T *y, int transpose, const float *Tball = nullptr);
// Block reflectors of the two-level FP32 factor (apply_qb.cu): T_b of every outer block
// from the blocks' Gram matrices and the inner panels' T, and Q^T y with them (returns
// 1 when not taken: Q y, or more than 160 x 296 rows)
int fl_block_t_f32(fastlsq_ctx *ctx, const float *Gall, const float *Tall, int64_t n, int nb, float *Tball);
int fl_apply_qb_f32(fastlsq_ctx *ctx, const float *F, int64_t ld, int64_t m_aug, int64_t n, const float *Tball,
                    float *y, int transpose);
template <typename TA, typename T>
int fl_copy_in(fastlsq_ctx *ctx, const TA *A, int64_t ldA, int64_t m, int64_t n, double mu,
               int64_t m_aug, const double *rhs, int64_t ld_rhs, int nrhs, T *F, int64_t ld);
template <typename T>
int fl_residual(fastlsq_ctx *ctx, const double *A, int64_t ldA, int64_t m, int64_t n, double mu,
                int64_t m_aug, const double *rhs, const double *beta, T *r_out, double *norm_out);
template <typename T>
int fl_extract_rhs(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t n, int r, T *out);
template <typename T>
int fl_to_f64(fastlsq_ctx *ctx, const T *src, int64_t n, double *dst, int add,
              const int *skip = nullptr);
template <typename T>
int fl_from_f64(fastlsq_ctx *ctx, const double *src, int64_t n, int64_t n_total, T *dst,
                const int *skip = nullptr);

// Register-resident FP32 panel of width 32 (panel_reg.cu); fits: rows per warp <= 24.
// With kp >= 0 the kernel first applies the panel at column kp (its reflectors in F,
// its T in Tprev) to this panel's columns, rows kp.. (the look-ahead update fused in).
// Returns 1 when the panel is too tall for registers, 2 when the fused form does not fit.
bool fl_panel_reg_fits(int64_t mp);
// Shared-memory panel of width 16 for tall FP32 panels (panel_tall.cu): 0 on launch,
// 1 when the panel is too short (the register kernels) or too tall for it.  With
// kp >= 0 the kernel first applies the previous panel (reflectors at columns kp = k - 16,
// T in Tprev) to this panel's columns, rows kp.. (the look-ahead update).
bool fl_panel_tall_fits(fastlsq_ctx *ctx, int64_t mp, bool fused);
int fl_panel_tall_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                      float *tau, float *Tblk, int64_t kp = -1, const float *Tprev = nullptr);
// Row-layout register panel (panel_row.cu), tried first by fl_panel_reg_f32 when the
// context's row_panel option is on: 1 = too tall, 2 = fused form does not fit.
int fl_panel_row_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                     float *tau, float *Tblk, int64_t kp, const float *Tprev);
bool fl_panel_row_fits(fastlsq_ctx *ctx, int64_t mp, bool fused);
bool fl_panel_reg_fused_fits(fastlsq_ctx *ctx, int64_t mp);
int fl_panel_reg_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                     float *tau, float *Tblk, int64_t kp = -1, const float *Tprev = nullptr);

// tcgen05 (TF32x3 split precision) trailing update fed by TMA; tc_update.cu.  ntot:
// columns of F.  Returns 1 when the tensor-core path does not take the shape (panel
// width other than 32, unaligned factor), the caller then runs the SIMT update.
int fl_trailing_tc_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int ncols,
                       int nb, int64_t nct, int64_t coff, int64_t ntot, const float *Tblk, int *counters);

// Outer-block trailing update on the tensor cores (three-part bf16 split), tc_block.cu:
// C <- H^T C for the block of nbk <= 128 columns at column k (inner panels of width nb,
// T factors from Tb on), C = F's columns k + nbk .. ntot.  Returns 1 when the shape is
// not taken (unaligned factor).  Gout (may be null) receives the block's Gram matrix
// V^T V, G[e * 128 + l] = v_l^T v_e for l, e < nbk.  With split_next the update pass of
// the next block's 128 columns runs on the caller's stream and the rest on the context's
// second auxiliary stream, to be joined by fl_block_join (the next call joins first).
int fl_block_update_f32(fastlsq_ctx *ctx, float *F, int64_t ld, int64_t k, int64_t m_aug, int nbk,
                        int64_t ntot, int nb, const float *Tb, float *Gout = nullptr, int split_next = 0);
int fl_block_join(fastlsq_ctx *ctx);

// TMA descriptor of the factor F (ld rows x ntot columns, column-major fp32) as a 2-D
// tensor with boxes of box_r rows x box_c columns, out-of-range elements read as zero
// (tc_update.cu); false when the driver's encoder is unavailable or rejects the shape
bool fl_encode_f32_map(CUtensorMap *m, const float *F, int64_t ld, int64_t ntot, uint32_t box_r, uint32_t box_c,
                       bool swizzle128);

// Thin Q of an FP64 factor: columns [col0, col0 + n) of F (ld rows, col0 >= n, F's
// first n columns the factor, T blocks Tall) set to Q [I_n; 0] (qr.cu)
int fl_form_q_f64(fastlsq_ctx *ctx, double *F, int64_t ld, int64_t m_aug, int64_t n, int nb, const double *Tall,
                  int64_t col0);

// Krylov refinement with the factor's R as preconditioner (refine.cu)
int fl_refine_cgls(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *rhs64, double *beta64,
                   int max_iter, double tol, double *norms_dev);
int fl_normal_pcg(fastlsq_ctx *ctx, const fastlsq_factor *f, const double *c64, double *v64,
                  int max_iter, double tol);

// triangular solve with R of type T (refine.cu): FP64 arithmetic, or for an FP32 factor
// FP32 (FL_ARITH_F32) or double-float (FL_ARITH_DF) arithmetic in the cluster kernel
constexpr int FL_ARITH_F32 = 1;
constexpr int FL_ARITH_DF = 2;
template <typename T>
int fl_trsv_grid(fastlsq_ctx *ctx, const T *F, int64_t ld, int64_t n, const double *y, double *x,
                 double *work, int transpose, const void *skip_scalars = nullptr, int arith = 0);

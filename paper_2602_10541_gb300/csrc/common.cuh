// Shared internals of libfastlsq (GB300, sm_103a): context, workspace, error
// handling and the operator parameter block passed to kernels by value.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/fastlsq.h"

// Kernel attributes (the dynamic shared-memory limit, non-portable cluster sizes) belong
// to the kernel's module in one device's context, so they are set once per device, not
// once per process.  Device ordinals past 63 set them on every call.
struct FlOncePerDevice {
    std::atomic<uint64_t> bits{0};
    bool pending(int dev) const
    {
        return dev < 0 || dev >= 64 || !((bits.load(std::memory_order_acquire) >> dev) & 1u);
    }
    void done(int dev)
    {
        if (dev >= 0 && dev < 64) bits.fetch_or(uint64_t(1) << dev, std::memory_order_acq_rel);
    }
};

// Trailing-update modes of the FP32 factorisation (values of FASTLSQ_OPT_TENSOR_CORE).
#define FL_TC_SIMT 0       // SIMT FP32, panel by panel
#define FL_TC_BLOCKED 1    // outer blocks of 128 columns on tcgen05, three-part bf16 split
#define FL_TC_PANEL 2      // panel by panel on tcgen05, TF32x3 split

#define FL_MAX_D 8
#define FL_MAX_TERMS 32
#define FL_MAX_PP 8
#define FL_MAX_FEAT 16384

// Device error flag codes (first one raised wins).
#define FL_DEVERR_NONFINITE 1
#define FL_DEVERR_BOUNDS 2
#define FL_DEVERR_TIMEOUT 3

struct fl_buffer {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Workspace slots (grow-only device buffers owned by the context).
enum fl_slot {
    FL_WS_PREFACTOR = 0,   // column prefactors P, Q and per-point multipliers
    FL_WS_PARTIAL,         // split-K / split-column partial sums
    FL_WS_VEC0,            // FP64 vectors for refinement
    FL_WS_VEC1,
    FL_WS_VEC2,
    FL_WS_SCALARS,         // small FP64 scratch (norms)
    FL_WS_NEWTON_J,        // Newton: FP32 Jacobian
    FL_WS_NEWTON_L64,      // Newton: FP64 linear operator rows
    FL_WS_NEWTON_H64,      // Newton: FP64 basis at interior rows
    FL_WS_NEWTON_VEC,      // Newton: vectors
    FL_WS_GRAM,            // panel Gram partials
    FL_WS_NORMS,           // residual norms for solve stats
    FL_WS_KRYLOV,          // Krylov refinement vectors and scalars
    FL_WS_APPLYQ,          // Q application partial sums
    FL_WS_SOLVE64,         // FP64 vectors of the triangular solves
    FL_WS_ZBUF,            // Z = T^T V^T C of the current trailing update
    FL_WS_COUNTERS,        // completion counters of the trailing-update column tiles
    FL_WS_VIMG,            // the panel's V as the tensor-core update's operand image
    FL_WS_WGRAD,           // row-chunk partial sums of the feature-weight gradient
    FL_WS_BLK_VY,          // outer-block update: V^T operand image (per 64-row chunk)
    FL_WS_BLK_VU,          // outer-block update: V operand image (per 128-row tile)
    FL_WS_BLK_Y,           // outer-block update: Y = V^T [V | C] split partials
    FL_WS_BLK_Z,           // outer-block update: Z operand image
    FL_WS_BLK_G,           // outer blocks' Gram matrices V_b^T V_b (for their block reflectors' T)
    FL_WS_COUNT
};

struct fl_prof_state {
    bool enabled = false;
    unsigned mask = 0;
    long long launches[FASTLSQ_K_COUNT] = {};
    std::vector<cudaEvent_t> ev[FASTLSQ_K_COUNT];   // start/end pairs
    size_t used[FASTLSQ_K_COUNT] = {};
    double ms[FASTLSQ_K_COUNT] = {};
};

struct fastlsq_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int max_smem_optin = 0;
    std::string last_error;
    fl_buffer ws[FL_WS_COUNT];
    int *d_flag = nullptr;          // device error flag (int)
    void *d_grid_bar = nullptr;     // grid barrier state (count, generation) of this context
    int use_tensor_core = 1;        // MIXED trailing updates: FL_TC_SIMT, FL_TC_BLOCKED or FL_TC_PANEL
    int panel_reg = 1;              // register-resident FP32 panel (width 32) where it fits
    int row_panel = 1;              // of which the row layout (one or two rows per thread)
    int lookahead = 1;              // panel p+1 beside the rest of panel p's update (on aux_stream)
    int fuse_next = 1;              // look-ahead: next panel applies the previous update itself
    int split_rows = 256;           // least rows per split of the SIMT trailing updates' Y pass
    int trsv32 = 1;                 // FP32 arithmetic in the triangular solves of classical refinement
    int inverse_thin_q = 1;         // inverse plans keep the thin Q of the interior rows
    int asm64_ctas_per_sm = 0;      // FP64 assembly: 0 one CTA per tile, k a persistent grid
    int krylov_df = 1;              // double-float preconditioner solves in CGLS / PCG (FP32 factors)
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t aux2_stream = nullptr;   // the rest of an outer block's update pass (look-ahead)
    cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
    int join2_pending = 0;                // ev_join2 recorded and not yet waited for
    cudaEvent_t refine_event = nullptr;   // waited on before reads of A_refine (caller's)
    double *eval_static = nullptr;  // device address of fastlsq_eval_noalloc's fixed scratch
    // Cody-Waite split of 2 pi for the FP32 argument reduction (host-derived)
    float cw2pi[3] = {0.f, 0.f, 0.f};
    fl_prof_state prof;
};

// Records CUDA events around the launches in its scope (when profiling is on) and
// counts one launch per kernel launched in the scope.
struct fl_prof_scope {
    fastlsq_ctx *ctx;
    int id;
    cudaEvent_t end = nullptr;
    fl_prof_scope(fastlsq_ctx *c, int kid, int n_launches = 1);
    ~fl_prof_scope();
};
#define FL_PROF(ctx, kid) fl_prof_scope _fl_prof_scope((ctx), (kid))
#define FL_PROF_N(ctx, kid, n) fl_prof_scope _fl_prof_scope((ctx), (kid), (n))

struct fastlsq_factor {
    fastlsq_ctx *ctx = nullptr;  // creating context (not dereferenced by _destroy)
    cudaStream_t stream = nullptr;
    int prec = 0;              // fastlsq_prec
    int64_t m = 0, n = 0;      // rows of A and features
    int64_t m_aug = 0, ld = 0; // factored rows (m + n when mu > 0), leading dimension
    double mu = 0.0;
    int nb = 32;
    void *F = nullptr;         // factor storage m_aug x n (float or double)
    void *tau = nullptr;       // n
    void *T = nullptr;         // (n / nb) blocks of nb x nb (column-major)
    void *Tb = nullptr;        // two-level factor: per outer block its 128 x 128 T_b (row-major)
    int has_tb = 0;            // Tb holds every outer block's T_b
    const double *A_refine = nullptr;
    int64_t ld_refine = 0;
    int tensor_core = 0;
};

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
int fl_fail(fastlsq_ctx *ctx, int code, const char *fmt, ...);
int fl_cuda(fastlsq_ctx *ctx, cudaError_t e, const char *what);
void *fl_ws(fastlsq_ctx *ctx, int slot, size_t bytes);   // nullptr on failure (error set)

#define FL_CHECK_LAUNCH(ctx, what)                                          \
    do {                                                                    \
        cudaError_t _e = cudaGetLastError();                                \
        if (_e != cudaSuccess) return fl_cuda((ctx), _e, (what));           \
    } while (0)

#define FL_TRY(expr)                                                        \
    do {                                                                    \
        int _rc = (expr);                                                   \
        if (_rc < 0) return _rc;                                            \
    } while (0)

__host__ __device__ __forceinline__ int64_t fl_min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t fl_max64(int64_t a, int64_t b) { return a > b ? a : b; }
static inline int64_t fl_cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t fl_round_up(int64_t a, int64_t b) { return fl_cdiv(a, b) * b; }

// ---------------------------------------------------------------------------
// Operator parameter block (by value into kernels)
// ---------------------------------------------------------------------------
struct fl_op_params {
    int d;
    int n_terms;
    int alpha[FL_MAX_TERMS][FL_MAX_D];
    double coef[FL_MAX_TERMS];
    int n_pp;
    int pp_alpha[FL_MAX_PP][FL_MAX_D];
    const double *pp_coef[FL_MAX_PP];
};

int fl_pack_op(fastlsq_ctx *ctx, const fastlsq_op *op, fl_op_params *out);

// Sums, on the device and in block order, the per-block partials part[blk * stride + q]
// (q < ncols, ncols <= 64) into part[nblk * stride + q], then copies them to host_out and
// synchronises the context's stream.  part must hold nblk + 1 rows of stride doubles.
int fl_reduce_blocks_to_host(fastlsq_ctx *ctx, double *part, int64_t nblk, int stride, int ncols,
                             double *host_out);

// Kernels / launchers implemented in the .cu files ---------------------------
int fl_prefactors(fastlsq_ctx *ctx, const fl_op_params &op, const double *W, int64_t n_feat,
                  double scale, double row_weight, double *pref);
int fl_launch_assemble_f32(fastlsq_ctx *ctx, const fl_op_params &op, const double *x,
                           int64_t n_rows, const double *W, const double *b, int64_t n_feat,
                           const double *pref, float *A, int64_t ldA, int64_t row_offset,
                           double row_weight);
int fl_launch_assemble_f64(fastlsq_ctx *ctx, const fl_op_params &op, const double *x,
                           int64_t n_rows, const double *W, const double *b, int64_t n_feat,
                           const double *pref, double *A, int64_t ldA, int64_t row_offset,
                           double row_weight);

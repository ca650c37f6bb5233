"""Thin Python binding of libfastlsq (include/fastlsq.h), argument marshalling only.

Each function has the name of the C entry point it calls.  Device arrays are
torch CUDA tensors (their data pointers are passed through); host arrays are
numpy arrays or Python sequences.  A column-major matrix with leading dimension
ld is represented by a contiguous torch tensor of shape (n_cols, ld): element
(i, j) is ``M[j, i]`` (see ``colmajor``).  Every step of the computation runs in
the library's CUDA kernels; nothing here computes.  A missing library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_lib = None

F32, F64 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
REFINE_CLASSICAL, REFINE_CGLS = 0, 1
RHS_SOURCE, RHS_EXACT, RHS_COEF, RHS_COEF_GRAD = 0, 1, 2, 3
POISSON_1D, HELMHOLTZ_2D, POISSON_5D, BRATU_2D, GAUSS_SOURCE_2D = 1, 2, 3, 4, 5
NLPOISSON_2D, NLHELMHOLTZ_2D = 6, 7
ALLEN_CAHN_1D, BURGERS_1D = 8, 9
VARCOEF_2D = 10
NL_NONE, NL_EXP, NL_CUBIC, NL_BURGERS = 0, 1, 2, 3

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double


class fastlsq_op(ctypes.Structure):
    _fields_ = [("d", _i32), ("n_terms", _i32), ("alpha", ctypes.POINTER(_i32)),
                ("coef", ctypes.POINTER(_dbl)), ("n_pp", _i32),
                ("pp_alpha", ctypes.POINTER(_i32)), ("pp_coef", ctypes.POINTER(_vp))]


class fastlsq_solve_stats(ctypes.Structure):
    _fields_ = [("refine_steps", _i32), ("nb", _i32), ("tensor_core", _i32), ("status", _i32),
                ("resid_norm", _dbl * 65)]


class fastlsq_newton_problem(ctypes.Structure):
    _fields_ = [("d", _i32), ("n_int", _i64), ("n_bc", _i64), ("x_int", _vp), ("x_bc", _vp),
                ("op", fastlsq_op), ("nl_kind", _i32), ("nl_lam", _dbl), ("bc_weight", _dbl),
                ("f", _vp), ("g", _vp)]


class fastlsq_newton_opts(ctypes.Structure):
    _fields_ = [("max_iter", _i32), ("tol", _dbl), ("mu", _dbl), ("armijo_c", _dbl),
                ("max_halvings", _i32), ("prec", _i32), ("max_refine", _i32), ("refine_tol", _dbl)]


class fastlsq_newton_stats(ctypes.Structure):
    _fields_ = [("iters", _i32), ("status", _i32), ("res_norm", _dbl * 65),
                ("step_rel", _dbl * 64), ("alpha", _dbl * 64)]


class fastlsq_inverse_instance(ctypes.Structure):
    _fields_ = [("n_int", _i64), ("n_bc", _i64), ("n_feat", _i64), ("n_sens", _i64),
                ("x_int", _vp), ("x_bc", _vp), ("W", _vp), ("b", _vp), ("sensors", _vp),
                ("y_obs", _vp), ("theta", _vp), ("beta", _vp), ("loss", _vp), ("dtheta", _vp)]


class fastlsq_inverse_opts(ctypes.Structure):
    _fields_ = [("prec", _i32), ("refine_iters", _i32), ("refine_tol", _dbl),
                ("adjoint_iters", _i32), ("adjoint_tol", _dbl), ("mu", _dbl), ("bc_weight", _dbl)]


_SIGNATURES = {
    "fastlsq_create": [ctypes.POINTER(_vp), ctypes.c_int, _vp],
    "fastlsq_destroy": [_vp],
    "fastlsq_set_stream": [_vp, _vp],
    "fastlsq_set_refine_event": [_vp, _vp],
    "fastlsq_last_error": [_vp],
    "fastlsq_sync": [_vp],
    "fastlsq_set_option": [_vp, ctypes.c_int, ctypes.c_int],
    "fastlsq_assemble": [_vp, ctypes.c_int, _vp, _i64, ctypes.POINTER(fastlsq_op), _dbl, _vp, _vp,
                         _i64, _dbl, _vp, _i64, _i64],
    "fastlsq_rhs": [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_dbl), _i32, _vp, _i64, _i32,
                    _dbl, _vp],
    "fastlsq_eval": [_vp, _vp, _i64, _i32, _vp, _vp, _i64, _dbl, _vp, _vp],
    "fastlsq_eval_op": [_vp, _vp, _i64, _i32, ctypes.POINTER(fastlsq_op), _vp, _vp, _i64, _dbl, _vp, _vp],
    "fastlsq_eval_noalloc": [_vp, _vp, _i64, _i32, _vp, _vp, _i64, _dbl, _vp, _vp],
    "fastlsq_eval_adjoint": [_vp, _vp, _i64, _i32, _vp, _vp, _i64, _dbl, _vp, _vp],
    "fastlsq_lstsq": [_vp, ctypes.c_int, _vp, ctypes.c_int, _i64, _i64, _i64, _dbl, _vp, _i32, _i64,
                      _vp, _i64, _vp, _i64, _i32, _i32, _dbl, ctypes.POINTER(_vp),
                      ctypes.POINTER(fastlsq_solve_stats)],
    "fastlsq_factor_solve": [_vp, _vp, _vp, _i32, _i64, _vp, _i64, _i32, _i32, _dbl,
                             ctypes.POINTER(fastlsq_solve_stats)],
    "fastlsq_factor_destroy": [_vp],
    "fastlsq_factor_get_r": [_vp, _vp, _vp, _i64],
    "fastlsq_factor_trsv": [_vp, _vp, _vp, _vp, _i32],
    "fastlsq_backward": [_vp, _vp, _vp, _vp, _vp, _vp, _i64, _i32, _dbl],
    "fastlsq_source_grad": [_vp, _vp, _i64, ctypes.POINTER(_dbl), _i32, _vp, ctypes.POINTER(_dbl)],
    "fastlsq_coef_grad": [_vp, _vp, _i64, ctypes.POINTER(fastlsq_op), _vp, _vp, _i64, _dbl, _vp,
                          _vp, _vp, _vp, ctypes.POINTER(_dbl)],
    "fastlsq_newton": [_vp, ctypes.POINTER(fastlsq_newton_problem), _vp, _vp, _i64, _dbl,
                       ctypes.POINTER(fastlsq_newton_opts), _vp,
                       ctypes.POINTER(fastlsq_newton_stats)],
    "fastlsq_newton_continuation": [_vp, ctypes.POINTER(fastlsq_newton_problem), _vp, _vp, _i64,
                                    _dbl, ctypes.POINTER(fastlsq_newton_opts), _i32,
                                    ctypes.POINTER(_dbl), _vp, ctypes.POINTER(fastlsq_newton_stats)],
    "fastlsq_weight_grad": [_vp, _vp, _i64, ctypes.POINTER(fastlsq_op), _dbl, _vp, _vp, _i64, _dbl,
                            _vp, _vp, _vp, _vp, _dbl, _dbl, _dbl, _vp, _vp],
    "fastlsq_bandwidth_grad": [_vp, _vp, _vp, _i64, _i32, _vp],
    "fastlsq_residual": [_vp, _vp, _i64, _i64, _i64, _vp, _vp, _vp],
    "fastlsq_inverse_batch": [_vp, ctypes.POINTER(fastlsq_inverse_instance), _i32,
                              ctypes.POINTER(fastlsq_op), _i32, ctypes.POINTER(fastlsq_inverse_opts)],
    "fastlsq_inverse_prepare": [_vp, ctypes.POINTER(fastlsq_inverse_instance), _i32,
                                ctypes.POINTER(fastlsq_op), _i32, ctypes.POINTER(fastlsq_inverse_opts),
                                ctypes.POINTER(_vp)],
    "fastlsq_inverse_eval": [_vp, _vp, _i32, _i32, _i32],
    "fastlsq_inverse_plan_destroy": [_vp],
    "fastlsq_selftest_wait": [_vp, _i32, _i64],
    "fastlsq_profile_enable": [_vp, ctypes.c_int],
    "fastlsq_profile_read": [_vp, ctypes.c_int, ctypes.POINTER(_i64), ctypes.POINTER(_dbl)],
}

KERNELS = ["prefactor", "assemble_f32", "assemble_f64", "rhs", "eval", "copy_in", "panel",
           "trail_simt", "trail_tc", "apply_q", "trsv", "residual", "vector", "newton", "adjoint",
           "krylov", "block_prep", "block_y", "block_u"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libfastlsq.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError("libfastlsq.so is not built: run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, args in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "fastlsq_last_error" else ctypes.c_int
    _lib = lib
    return lib


class FastLSQError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fastlsq error {code}: {msg}")
        self.code = code


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """fastlsq_create / fastlsq_destroy around torch's current CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.fastlsq_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise FastLSQError(rc, "fastlsq_create failed")
        self.handle = h

    def check(self, rc, allow_warnings=True):
        if rc < 0 or (rc > 0 and not allow_warnings):
            msg = self.lib.fastlsq_last_error(self.handle)
            raise FastLSQError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fastlsq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


OPT_TENSOR_CORE = 0
OPT_REGISTER_PANEL = 1
OPT_LOOKAHEAD = 2
OPT_TRSV_FP32 = 3
OPT_FUSED_LOOKAHEAD = 4
OPT_ROW_PANEL = 5
OPT_SPLIT_ROWS = 6
OPT_INVERSE_THIN_Q = 7
OPT_FP64_ASSEMBLY_CTAS = 8
OPT_KRYLOV_DF = 9


def fastlsq_set_option(ctx, option, value):
    return ctx.check(ctx.lib.fastlsq_set_option(ctx.handle, int(option), int(value)))


def fastlsq_set_stream(ctx, stream):
    """Queue the context's later work on `stream` (a torch.cuda.Stream)."""
    ctx.stream = stream
    return ctx.check(ctx.lib.fastlsq_set_stream(ctx.handle, ctypes.c_void_p(stream.cuda_stream)))


def fastlsq_set_refine_event(ctx, event):
    """Reads of a factor's FP64 operator wait for `event` (a torch.cuda.Event that has
    been recorded; None removes the wait)."""
    h = None if event is None else ctypes.c_void_p(event.cuda_event)
    return ctx.check(ctx.lib.fastlsq_set_refine_event(ctx.handle, h))


def colmajor(n_rows, n_cols, dtype, device, ld=None, zero=False):
    """Allocate a column-major matrix as a (n_cols, ld) torch tensor (ld >= n_rows,
    rounded up to a multiple of 4 by default)."""
    import torch
    ld = ld or ((n_rows + 3) // 4) * 4
    fn = torch.zeros if zero else torch.empty
    return fn((n_cols, ld), dtype=dtype, device=device)


class Op:
    """Operator terms sum_t coef[t] D^{alpha_t} plus optional per-point terms; holds
    the host arrays the fastlsq_op struct points to."""

    def __init__(self, alpha, coef, pp_alpha=None, pp_coef=None):
        self.alpha = np.ascontiguousarray(np.atleast_2d(alpha), dtype=np.int32)
        self.coef = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
        self.d = self.alpha.shape[1]
        self.pp_alpha = (np.ascontiguousarray(np.atleast_2d(pp_alpha), dtype=np.int32)
                         if pp_alpha is not None else None)
        self.pp_tensors = list(pp_coef) if pp_coef is not None else []
        n_pp = len(self.pp_tensors)
        self._pp_ptrs = (ctypes.c_void_p * max(1, n_pp))(*[t.data_ptr() for t in self.pp_tensors])
        self.struct = fastlsq_op(
            self.d, self.alpha.shape[0], self.alpha.ctypes.data_as(ctypes.POINTER(_i32)),
            self.coef.ctypes.data_as(ctypes.POINTER(_dbl)), n_pp,
            self.pp_alpha.ctypes.data_as(ctypes.POINTER(_i32)) if n_pp else None,
            ctypes.cast(self._pp_ptrs, ctypes.POINTER(_vp)) if n_pp else None)

    @staticmethod
    def identity(d):
        return Op(np.zeros((1, d), np.int32), [1.0])


def fastlsq_assemble(ctx, dtype, x, op, row_weight, W, b, scale, A, row_offset=0, n_rows=None):
    n_rows = x.shape[0] if n_rows is None else n_rows
    if n_rows > x.shape[0] or x.shape[1] != op.d or W.shape[1] != op.d or b.numel() < W.shape[0]:
        raise ValueError("fastlsq_assemble: array shapes do not match the sizes")
    return ctx.check(ctx.lib.fastlsq_assemble(
        ctx.handle, dtype, _ptr(x), n_rows, ctypes.byref(op.struct), float(row_weight), _ptr(W),
        _ptr(b), W.shape[0], float(scale), _ptr(A), A.shape[1], row_offset))


def fastlsq_rhs(ctx, problem, kind, params, x, weight, out):
    p = np.ascontiguousarray(params if params is not None else [], dtype=np.float64).reshape(-1)
    pp = p.ctypes.data_as(ctypes.POINTER(_dbl)) if p.size else None
    return ctx.check(ctx.lib.fastlsq_rhs(ctx.handle, problem, kind, pp, p.size, _ptr(x),
                                         x.shape[0], x.shape[1], float(weight), _ptr(out)))


def fastlsq_eval(ctx, x, W, b, scale, beta, u):
    return ctx.check(ctx.lib.fastlsq_eval(ctx.handle, _ptr(x), x.shape[0], x.shape[1], _ptr(W),
                                          _ptr(b), W.shape[0], float(scale), _ptr(beta), _ptr(u)))


def fastlsq_eval_op(ctx, x, op, W, b, scale, beta, u):
    """(L u)(x_e) for the operator `op` (an Op without per-point terms)."""
    return ctx.check(ctx.lib.fastlsq_eval_op(ctx.handle, _ptr(x), x.shape[0], x.shape[1],
                                             ctypes.byref(op.struct), _ptr(W), _ptr(b), W.shape[0],
                                             float(scale), _ptr(beta), _ptr(u)))


def fastlsq_eval_noalloc(ctx, x, W, b, scale, beta, u):
    """fastlsq_eval with the scratch in the library's fixed device array (no allocation)."""
    return ctx.check(ctx.lib.fastlsq_eval_noalloc(ctx.handle, _ptr(x), x.shape[0], x.shape[1], _ptr(W),
                                                  _ptr(b), W.shape[0], float(scale), _ptr(beta), _ptr(u)))


def fastlsq_eval_adjoint(ctx, x, W, b, scale, g, grad_beta):
    return ctx.check(ctx.lib.fastlsq_eval_adjoint(ctx.handle, _ptr(x), x.shape[0], x.shape[1],
                                                  _ptr(W), _ptr(b), W.shape[0], float(scale),
                                                  _ptr(g), _ptr(grad_beta)))


def fastlsq_lstsq(ctx, prec, A, n_rows, mu, rhs, beta, A_refine=None, max_refine=0, keep=False,
                  stats=False, refine_mode=REFINE_CLASSICAL, refine_tol=1e-10):
    """A: (n_feat, ldA) float32/float64 column-major; rhs: (nrhs, ld_rhs) float64;
    beta: (nrhs, n_feat) float64.  Returns (status, factor handle or None, stats or None)."""
    import torch
    a_dtype = F64 if A.dtype == torch.float64 else F32
    n_feat = A.shape[0]
    handle = ctypes.c_void_p()
    st = fastlsq_solve_stats() if stats else None
    nrhs = 0 if rhs is None else rhs.shape[0]
    rc = ctx.lib.fastlsq_lstsq(
        ctx.handle, prec, _ptr(A), a_dtype, A.shape[1], n_rows, n_feat, float(mu), _ptr(rhs),
        nrhs, rhs.shape[1] if nrhs else 0, _ptr(beta), beta.shape[1] if nrhs else 0, _ptr(A_refine),
        A_refine.shape[1] if A_refine is not None else 0, int(max_refine), int(refine_mode),
        float(refine_tol), ctypes.byref(handle) if keep else None,
        ctypes.byref(st) if stats else None)
    ctx.check(rc)
    return rc, (handle if keep else None), st


def fastlsq_factor_solve(ctx, factor, rhs, beta, max_refine=0, stats=False,
                         refine_mode=REFINE_CLASSICAL, refine_tol=1e-10):
    st = fastlsq_solve_stats() if stats else None
    rc = ctx.lib.fastlsq_factor_solve(ctx.handle, factor, _ptr(rhs), rhs.shape[0], rhs.shape[1],
                                      _ptr(beta), beta.shape[1], int(max_refine), int(refine_mode),
                                      float(refine_tol), ctypes.byref(st) if stats else None)
    ctx.check(rc)
    return rc, st


def fastlsq_factor_get_r(ctx, factor, R):
    """R: (n_feat, ld >= n_feat) float64 column-major tensor."""
    return ctx.check(ctx.lib.fastlsq_factor_get_r(ctx.handle, factor, _ptr(R), R.shape[1]))


def fastlsq_factor_trsv(ctx, factor, y, x, transpose=False):
    return ctx.check(ctx.lib.fastlsq_factor_trsv(ctx.handle, factor, _ptr(y), _ptr(x),
                                                 1 if transpose else 0))


def fastlsq_factor_destroy(ctx, factor):
    return ctx.lib.fastlsq_factor_destroy(factor)


def fastlsq_backward(ctx, factor, grad_beta, v, grad_rhs=None, A_op=None, max_iter=0, tol=1e-12):
    return ctx.check(ctx.lib.fastlsq_backward(ctx.handle, factor, _ptr(grad_beta), _ptr(v),
                                              _ptr(grad_rhs), _ptr(A_op),
                                              A_op.shape[1] if A_op is not None else 0,
                                              int(max_iter), float(tol)))


def fastlsq_source_grad(ctx, x, theta, w):
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    out = np.zeros(th.size)
    ctx.check(ctx.lib.fastlsq_source_grad(ctx.handle, _ptr(x), x.shape[0],
                                          th.ctypes.data_as(ctypes.POINTER(_dbl)), th.size // 4,
                                          _ptr(w), out.ctypes.data_as(ctypes.POINTER(_dbl))))
    return out


def fastlsq_coef_grad(ctx, x, op, W, b, scale, r, Av, v, beta):
    out = np.zeros(op.alpha.shape[0])
    ctx.check(ctx.lib.fastlsq_coef_grad(ctx.handle, _ptr(x), x.shape[0], ctypes.byref(op.struct),
                                        _ptr(W), _ptr(b), W.shape[0], float(scale), _ptr(r),
                                        _ptr(Av), _ptr(v), _ptr(beta),
                                        out.ctypes.data_as(ctypes.POINTER(_dbl))))
    return out


def fastlsq_weight_grad(ctx, x, op, row_weight, W, b, scale, r, beta, gW, gb=None, v=None, Av=None,
                        c_v=1.0, c_rb=0.0, c_av=-1.0):
    """Accumulate the feature-weight (gW [n_feat][d]) and bias (gb) gradients of one row block."""
    return ctx.check(ctx.lib.fastlsq_weight_grad(
        ctx.handle, _ptr(x), x.shape[0], ctypes.byref(op.struct), float(row_weight), _ptr(W),
        _ptr(b), W.shape[0], float(scale), _ptr(r), _ptr(beta), _ptr(v), _ptr(Av), float(c_v),
        float(c_rb), float(c_av), _ptr(gW), _ptr(gb)))


def fastlsq_bandwidth_grad(ctx, gW, W_hat, out):
    """out [d*d + 1] (device): sum_j gW[j][a] W_hat[j][c], then the trace."""
    return ctx.check(ctx.lib.fastlsq_bandwidth_grad(ctx.handle, _ptr(gW), _ptr(W_hat), gW.shape[0],
                                                    gW.shape[1], _ptr(out)))


def fastlsq_residual(ctx, A, m, beta, rhs, r):
    """r = rhs - A beta for the FP64 operator A ([n][ld] storage of an m x n column-major matrix)."""
    return ctx.check(ctx.lib.fastlsq_residual(ctx.handle, _ptr(A), A.shape[1], m, A.shape[0], _ptr(beta),
                                              _ptr(rhs), _ptr(r)))


def fastlsq_newton(ctx, x_int, x_bc, op, nl_kind, nl_lam, bc_weight, f, g, W, b, scale, beta,
                   max_iter=15, tol=1e-10, mu=1e-10, armijo_c=1e-4, max_halvings=20,
                   prec=PREC_MIXED, max_refine=30, refine_tol=1e-10):
    prob = fastlsq_newton_problem(x_int.shape[1], x_int.shape[0], x_bc.shape[0], x_int.data_ptr(),
                                  x_bc.data_ptr(), op.struct, nl_kind, float(nl_lam),
                                  float(bc_weight), f.data_ptr(), g.data_ptr())
    opts = fastlsq_newton_opts(max_iter, float(tol), float(mu), float(armijo_c), max_halvings,
                               prec, max_refine, float(refine_tol))
    st = fastlsq_newton_stats()
    rc = ctx.lib.fastlsq_newton(ctx.handle, ctypes.byref(prob), _ptr(W), _ptr(b), W.shape[0],
                                float(scale), ctypes.byref(opts), _ptr(beta), ctypes.byref(st))
    ctx.check(rc)
    return rc, st


def fastlsq_newton_continuation(ctx, x_int, x_bc, op, stage_coef, nl_kind, nl_lam, bc_weight, f,
                                g, W, b, scale, beta, max_iter=12, tol=1e-10, mu=1e-10,
                                armijo_c=1e-4, max_halvings=20, prec=PREC_MIXED, max_refine=30,
                                refine_tol=1e-10):
    """stage_coef: [n_stages][op's n_terms] coefficients per stage.  Returns (status,
    [stats per stage])."""
    sc = np.ascontiguousarray(stage_coef, dtype=np.float64).reshape(-1, op.alpha.shape[0])
    prob = fastlsq_newton_problem(x_int.shape[1], x_int.shape[0], x_bc.shape[0], x_int.data_ptr(),
                                  x_bc.data_ptr(), op.struct, nl_kind, float(nl_lam),
                                  float(bc_weight), f.data_ptr(), g.data_ptr())
    opts = fastlsq_newton_opts(max_iter, float(tol), float(mu), float(armijo_c), max_halvings,
                               prec, max_refine, float(refine_tol))
    st = (fastlsq_newton_stats * sc.shape[0])()
    rc = ctx.lib.fastlsq_newton_continuation(ctx.handle, ctypes.byref(prob), _ptr(W), _ptr(b),
                                             W.shape[0], float(scale), ctypes.byref(opts),
                                             sc.shape[0], sc.ctypes.data_as(ctypes.POINTER(_dbl)),
                                             _ptr(beta), st)
    ctx.check(rc)
    return rc, list(st)


def fastlsq_profile_enable(ctx, classes=None):
    """classes: None = every kernel class, [] = stop recording, or a list of names."""
    if classes is None:
        mask = -1
    else:
        mask = 0
        for c in classes:
            mask |= 1 << KERNELS.index(c)
    return ctx.check(ctx.lib.fastlsq_profile_enable(ctx.handle, mask))


def fastlsq_profile_read(ctx):
    """{kernel class: (launches, total device ms)} since the last reset."""
    out = {}
    for k, name in enumerate(KERNELS):
        n = _i64(0)
        ms = _dbl(0.0)
        ctx.check(ctx.lib.fastlsq_profile_read(ctx.handle, k, ctypes.byref(n), ctypes.byref(ms)))
        out[name] = (int(n.value), float(ms.value))
    return out


def fastlsq_selftest_wait(ctx, which, budget_cycles):
    """Queue a kernel whose bounded wait (0: mbarrier, 1: grid barrier) runs out."""
    return ctx.check(ctx.lib.fastlsq_selftest_wait(ctx.handle, which, int(budget_cycles)))


def fastlsq_sync(ctx):
    """Wait for the context's stream and report a device-side error flag (raises)."""
    return ctx.check(ctx.lib.fastlsq_sync(ctx.handle))


def _inverse_instances(instances):
    arr = (fastlsq_inverse_instance * len(instances))()
    for q, d in enumerate(instances):
        arr[q] = fastlsq_inverse_instance(
            d["x_int"].shape[0], d["x_bc"].shape[0], d["W"].shape[0], d["sensors"].shape[0],
            d["x_int"].data_ptr(), d["x_bc"].data_ptr(), d["W"].data_ptr(), d["b"].data_ptr(),
            d["sensors"].data_ptr(), d["y_obs"].data_ptr(), d["theta"].data_ptr(),
            d["beta"].data_ptr(), d["loss"].data_ptr(), d["dtheta"].data_ptr())
    return arr


class InversePlan:
    """fastlsq_inverse_prepare / fastlsq_inverse_plan_destroy: the instances' factors
    and sensor matrices, kept for repeated evaluations (the instance tensors must stay
    alive and at the same addresses while the plan is used)."""

    def __init__(self, ctx, instances, op, n_src, mu=1e-10, bc_weight=100.0):
        self.ctx = ctx
        self.instances = list(instances)
        arr = _inverse_instances(self.instances)
        opts = fastlsq_inverse_opts(PREC_FP64, 0, 0.0, 0, 0.0, float(mu), float(bc_weight))
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.fastlsq_inverse_prepare(ctx.handle, arr, len(self.instances), ctypes.byref(op.struct),
                                                  n_src, ctypes.byref(opts), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.fastlsq_inverse_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fastlsq_inverse_prepare(ctx, instances, op, n_src, mu=1e-10, bc_weight=100.0):
    return InversePlan(ctx, instances, op, n_src, mu=mu, bc_weight=bc_weight)


def fastlsq_inverse_eval(ctx, plan, threads=256, ctas_per_sm=1, cluster=1):
    """One gradient evaluation of every instance of the plan (one persistent launch of
    clusters of `cluster` CTAs, one cluster per instance at a time)."""
    return ctx.check(ctx.lib.fastlsq_inverse_eval(ctx.handle, plan.handle, threads, ctas_per_sm, cluster))


def fastlsq_inverse_batch(ctx, instances, op, n_src, prec=PREC_MIXED, refine_iters=64,
                          refine_tol=1e-13, adjoint_iters=64, adjoint_tol=1e-13, mu=1e-10,
                          bc_weight=100.0):
    """instances: sequence of dicts with device tensors x_int, x_bc, W, b, sensors, y_obs,
    theta and output tensors beta, loss (1), dtheta (4 n_src)."""
    arr = (fastlsq_inverse_instance * len(instances))()
    for q, d in enumerate(instances):
        arr[q] = fastlsq_inverse_instance(
            d["x_int"].shape[0], d["x_bc"].shape[0], d["W"].shape[0], d["sensors"].shape[0],
            d["x_int"].data_ptr(), d["x_bc"].data_ptr(), d["W"].data_ptr(), d["b"].data_ptr(),
            d["sensors"].data_ptr(), d["y_obs"].data_ptr(), d["theta"].data_ptr(),
            d["beta"].data_ptr(), d["loss"].data_ptr(), d["dtheta"].data_ptr())
    opts = fastlsq_inverse_opts(prec, refine_iters, float(refine_tol), adjoint_iters,
                                float(adjoint_tol), float(mu), float(bc_weight))
    return ctx.check(ctx.lib.fastlsq_inverse_batch(ctx.handle, arr, len(instances),
                                                   ctypes.byref(op.struct), n_src,
                                                   ctypes.byref(opts)))

"""FP64 CPU oracle for the FastLSQ hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The GPU product path never calls it; it shares no code
with the CUDA sources.  The arithmetic lives in ``oracle.c`` (plain C, double
precision, no BLAS); this module compiles it with gcc on first use and exposes
numpy-friendly wrappers.

Every function is pinned by the CPU tests (``tests/test_oracle_*.py``) against
closed forms, finite differences, brute force or an independent solver; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Problem ids of orc_problem_source / orc_problem_exact (manufactured problems).
POISSON_1D = 1
HELMHOLTZ_2D = 2
POISSON_5D = 3
BRATU_2D = 4
GAUSS_SOURCE_2D = 5
NLPOISSON_2D = 6
NLHELMHOLTZ_2D = 7
ALLEN_CAHN_1D = 8
BURGERS_1D = 9
VARCOEF_2D = 10

NL_NONE, NL_EXP, NL_CUBIC, NL_BURGERS = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
           "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.c_long


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_assemble.argtypes = [_D, _L, ctypes.c_int, ctypes.c_int, _I, _D, _D,
                                     ctypes.c_double, _D, _D, _L, ctypes.c_double, _D, _L]
        lib.orc_eval_u.argtypes = [_D, _L, ctypes.c_int, _D, _D, _L, ctypes.c_double, _D, _D]
        lib.orc_qr.argtypes = [_D, _L, _L, _L, _D]
        lib.orc_apply_qt.argtypes = [_D, _L, _L, _L, _D, _D, ctypes.c_int, _L]
        lib.orc_backsolve.argtypes = [_D, _L, _L, _D]
        lib.orc_forwardsolve_rt.argtypes = [_D, _L, _L, _D]
        lib.orc_lstsq.argtypes = [_D, _L, _L, _L, ctypes.c_double, _D, ctypes.c_int, _D]
        lib.orc_lstsq.restype = ctypes.c_int
        lib.orc_problem_exact.argtypes = [ctypes.c_int, _D, _L, ctypes.c_int, _D, _D]
        lib.orc_problem_source.argtypes = [ctypes.c_int, _D, _L, ctypes.c_int, _D,
                                           ctypes.c_int, _D]
        lib.orc_gauss_source_grad.argtypes = [_D, _L, _D, ctypes.c_int, _D, _D]
        lib.orc_newton.argtypes = [_D, _L, _D, _L, ctypes.c_int, ctypes.c_int, _I, _D,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D,
                                   _D, _D, _L, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _I, _D]
        lib.orc_newton.restype = ctypes.c_int
        lib.orc_inverse_adjoint.argtypes = [_D, _L, _L, _L, ctypes.c_double, _D, _D, _L, _L,
                                            _D, _D, _D, _D, _D, _D, _D]
        lib.orc_inverse_adjoint.restype = ctypes.c_int
        lib.orc_term_coef_grad.argtypes = [_D, _L, ctypes.c_int, _I, _D, _D, _L,
                                           ctypes.c_double, _D, _D, _D, _D]
        lib.orc_term_coef_grad.restype = ctypes.c_double
        lib.orc_problem_coef.argtypes = [ctypes.c_int, ctypes.c_int, _D, _L, ctypes.c_int, _D, _D]
        lib.orc_weight_grad.argtypes = [_D, _L, ctypes.c_int, ctypes.c_int, _I, _D,
                                        ctypes.c_double, _D, _D, _L, ctypes.c_double, _D, _D,
                                        _D, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _D, _D]
        _lib = lib
        return lib


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def assemble(x, alpha, coef, W, b, scale, row_weight=1.0, coef_pt=None):
    """A (n_rows x n_feat, returned C-contiguous as [n_feat][n_rows] transposed view
    i.e. a numpy array of shape (n_rows, n_feat)) of the operator given by
    terms (alpha [n_terms][d], coef [n_terms]); see orc_assemble."""
    lib = _load()
    x = _f64(np.atleast_2d(x))
    n_rows, d = x.shape
    W = _f64(W).reshape(-1, d)
    b = _f64(b)
    alpha = _i32(alpha).reshape(-1, d)
    coef = _f64(coef)
    n_feat = W.shape[0]
    out = np.zeros((n_feat, n_rows), dtype=np.float64)   # column-major A
    cpt = None if coef_pt is None else _f64(coef_pt).reshape(alpha.shape[0], n_rows)
    lib.orc_assemble(_d(x), n_rows, d, alpha.shape[0], _i(alpha), _d(coef),
                     None if cpt is None else _d(cpt), float(row_weight),
                     _d(W), _d(b), n_feat, float(scale), _d(out), n_rows)
    return out.T


def eval_u(x, W, b, scale, beta):
    lib = _load()
    x = _f64(np.atleast_2d(x))
    n, d = x.shape
    W = _f64(W).reshape(-1, d)
    out = np.zeros(n)
    lib.orc_eval_u(_d(x), n, d, _d(W), _d(_f64(b)), W.shape[0], float(scale),
                   _d(_f64(beta)), _d(out))
    return out


def qr(A):
    """In-place style Householder QR of a copy of A; returns (packed [m x n] array
    in column-major storage exposed as (m, n), tau)."""
    lib = _load()
    m, n = A.shape
    packed = np.array(A, dtype=np.float64, order="F")
    tau = np.zeros(n)
    lib.orc_qr(_d(packed), m, n, m, _d(tau))
    return packed, tau


def apply_qt(packed, tau, y):
    lib = _load()
    m, n = packed.shape
    packed = np.asfortranarray(packed)
    y = np.array(y, dtype=np.float64, order="F")
    if y.ndim == 1:
        lib.orc_apply_qt(_d(packed), m, n, m, _d(tau), _d(y), 1, m)
    else:
        lib.orc_apply_qt(_d(packed), m, n, m, _d(tau), _d(y), y.shape[1], m)
    return y


def backsolve(packed, y):
    lib = _load()
    m, n = packed.shape
    packed = np.asfortranarray(packed)
    y = np.array(y[:n], dtype=np.float64)
    lib.orc_backsolve(_d(packed), n, m, _d(y))
    return y


def lstsq(A, rhs, mu=0.0):
    """beta = argmin ||A beta - rhs||^2 + mu ||beta||^2 (rhs: (m,) or (m, nrhs))."""
    lib = _load()
    A = np.asfortranarray(A, dtype=np.float64)
    m, n = A.shape
    rhs = np.asfortranarray(rhs, dtype=np.float64)
    nrhs = 1 if rhs.ndim == 1 else rhs.shape[1]
    beta = np.zeros((n, nrhs), order="F") if rhs.ndim == 2 else np.zeros(n)
    rc = lib.orc_lstsq(_d(A), m, n, m, float(mu), _d(rhs), nrhs, _d(beta))
    if rc != 0:
        raise MemoryError("orc_lstsq")
    return beta


def problem_coef(prob, comp, x, params=()):
    """Variable coefficient nu (comp = -1) or d nu / d x_comp at points (orc_problem_coef)."""
    lib = _load()
    x = _f64(np.atleast_2d(x))
    n, d = x.shape
    p = _f64(np.asarray(params, dtype=np.float64).reshape(-1) if len(params) else np.zeros(1))
    out = np.zeros(n)
    lib.orc_problem_coef(int(prob), int(comp), _d(x), n, d, _d(p), _d(out))
    return out


def problem_exact(prob, x, params=()):
    lib = _load()
    x = _f64(np.atleast_2d(x))
    n, d = x.shape
    p = _f64(np.asarray(params, dtype=np.float64).reshape(-1) if len(params) else np.zeros(1))
    out = np.zeros(n)
    lib.orc_problem_exact(int(prob), _d(x), n, d, _d(p), _d(out))
    return out


def problem_source(prob, x, params=()):
    lib = _load()
    x = _f64(np.atleast_2d(x))
    n, d = x.shape
    params = np.asarray(params, dtype=np.float64).reshape(-1)
    p = _f64(params if params.size else np.zeros(1))
    out = np.zeros(n)
    lib.orc_problem_source(int(prob), _d(x), n, d, _d(p), int(params.size), _d(out))
    return out


def gauss_source_grad(x, theta, w):
    lib = _load()
    x = _f64(np.atleast_2d(x))
    theta = _f64(theta).reshape(-1)
    out = np.zeros(theta.size)
    lib.orc_gauss_source_grad(_d(x), x.shape[0], _d(theta), theta.size // 4, _d(_f64(w)),
                              _d(out))
    return out


def newton(x_int, x_bc, alpha, coef, nl_kind, nl_lam, bc_weight, f, g, W, b, scale,
           mu, max_iter, tol, armijo_c=1e-4, max_halvings=20, beta0=None):
    """Newton-Raphson (orc_newton).  Returns (beta, status, iters, residual history)."""
    lib = _load()
    x_int = _f64(np.atleast_2d(x_int))
    x_bc = _f64(np.atleast_2d(x_bc))
    d = x_int.shape[1]
    W = _f64(W).reshape(-1, d)
    n_feat = W.shape[0]
    alpha = _i32(alpha).reshape(-1, d)
    beta = np.zeros(n_feat) if beta0 is None else np.array(beta0, dtype=np.float64)
    iters = ctypes.c_int(0)
    hist = np.zeros(max_iter + 1)
    st = lib.orc_newton(_d(x_int), x_int.shape[0], _d(x_bc), x_bc.shape[0], d,
                        alpha.shape[0], _i(alpha), _d(_f64(coef)), int(nl_kind), float(nl_lam),
                        float(bc_weight), _d(_f64(f)), _d(_f64(g)), _d(W), _d(_f64(b)),
                        n_feat, float(scale), float(mu), int(max_iter), float(tol),
                        float(armijo_c), int(max_halvings), _d(beta), ctypes.byref(iters),
                        _d(hist))
    if st < 0:
        raise MemoryError("orc_newton")
    return beta, st, iters.value, hist[: iters.value + 1]


def inverse_adjoint(A, rhs, Hs, y_obs, mu):
    """Forward map + adjoint of Sec. 3.8 (orc_inverse_adjoint).  Returns a dict."""
    lib = _load()
    A = np.asfortranarray(A, dtype=np.float64)
    m, n = A.shape
    Hs = np.asfortranarray(Hs, dtype=np.float64)
    ns = Hs.shape[0]
    beta, u_s, v = np.zeros(n), np.zeros(ns), np.zeros(n)
    grad_rhs, resid = np.zeros(m), np.zeros(m)
    loss = ctypes.c_double(0.0)
    rc = lib.orc_inverse_adjoint(_d(A), m, n, m, float(mu), _d(_f64(rhs)), _d(Hs), ns, ns,
                                 _d(_f64(y_obs)), _d(beta), _d(u_s), ctypes.byref(loss),
                                 _d(v), _d(grad_rhs), _d(resid))
    if rc != 0:
        raise MemoryError("orc_inverse_adjoint")
    return dict(beta=beta, u_s=u_s, loss=loss.value, v=v, grad_rhs=grad_rhs, resid=resid)


def term_coef_grad(x_int, alpha_t, W, b, scale, r, Av, v, beta):
    lib = _load()
    x_int = _f64(np.atleast_2d(x_int))
    n_int, d = x_int.shape
    W = _f64(W).reshape(-1, d)
    return lib.orc_term_coef_grad(_d(x_int), n_int, d, _i(_i32(alpha_t)), _d(W), _d(_f64(b)),
                                  W.shape[0], float(scale), _d(_f64(r)), _d(_f64(Av)),
                                  _d(_f64(v)), _d(_f64(beta)))


def weight_grad(x, alpha, coef, row_weight, W, b, scale, r, beta, v=None, Av=None, c_v=1.0,
                c_rb=0.0, c_av=-1.0):
    """Feature-weight and bias gradients of the bilinear adjoint form (orc_weight_grad).
    Returns (gW [n_feat][d], gb [n_feat])."""
    lib = _load()
    x = _f64(np.atleast_2d(x))
    n, d = x.shape
    W = _f64(W).reshape(-1, d)
    alpha = _i32(alpha).reshape(-1, d)
    gW = np.zeros_like(W)
    gb = np.zeros(W.shape[0])
    nul = ctypes.cast(None, _D)
    lib.orc_weight_grad(_d(x), n, d, alpha.shape[0], _i(alpha), _d(_f64(coef)), float(row_weight),
                        _d(W), _d(_f64(b)), W.shape[0], float(scale), _d(_f64(r)), _d(_f64(beta)),
                        nul if v is None else _d(_f64(v)), nul if Av is None else _d(_f64(Av)),
                        float(c_v), float(c_rb), float(c_av), _d(gW), _d(gb))
    return gW, gb

"""torch.autograd.Function wrappers over the C ABI (Sec. 2.5: gradients flow through
the pre-factored solve; Sec. 3.8: each evaluation costs two triangular solves).

``Factorization`` checkpoints the QR factors of the operator once;
``solve(rhs)`` is beta = R^{-1} Q^T [rhs; 0] and its backward is
``fastlsq_backward`` (v = R^{-1} R^{-T} grad_beta, grad_rhs = A v);
``gauss_source(theta)`` is the Gaussian heat source s(x; theta) with backward
``fastlsq_source_grad``; ``evaluate(beta)`` is u at points with backward
``fastlsq_eval_adjoint``.  PyTorch only carries tensors and the tape.
"""
from __future__ import annotations

import numpy as np
import torch

from . import fastlsq as fl


class Factorization:
    """Checkpointed QR factors of A (n_rows x n_feat, column-major (n_feat, ld) tensor)
    with Tikhonov mu; A_op is the FP64 operator used for grad_rhs = A v (and for
    refinement when prec is MIXED)."""

    def __init__(self, ctx, A, n_rows, mu, prec=fl.PREC_FP64, A_op=None, max_refine=0,
                 refine_mode=fl.REFINE_CGLS, refine_tol=1e-13, adjoint_iters=0, adjoint_tol=1e-13):
        self.ctx, self.n_rows, self.mu, self.prec = ctx, n_rows, mu, prec
        self.refine_mode, self.refine_tol = refine_mode, refine_tol
        self.adjoint_iters, self.adjoint_tol = adjoint_iters, adjoint_tol
        self.n_feat = A.shape[0]
        self.A_op = A_op if A_op is not None else (A if A.dtype == torch.float64 else None)
        self.max_refine = max_refine
        _, self.handle, _ = fl.fastlsq_lstsq(ctx, prec, A, n_rows, mu, None, None,
                                             A_refine=self.A_op, max_refine=0, keep=True)
        self.device = A.device

    def solve(self, rhs):
        return _Solve.apply(rhs, self)

    def close(self):
        # the factor's memory belongs to the device pool; once the context is gone
        # (interpreter shutdown) it is released with the process
        if self.handle is not None and getattr(self.ctx, "handle", None):
            fl.fastlsq_factor_destroy(self.ctx, self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(actx, rhs, fac):
        ld = ((fac.n_rows + 3) // 4) * 4
        r = torch.zeros((1, ld), dtype=torch.float64, device=fac.device)
        r[0, : fac.n_rows] = rhs
        beta = torch.empty((1, fac.n_feat), dtype=torch.float64, device=fac.device)
        fl.fastlsq_factor_solve(fac.ctx, fac.handle, r, beta, max_refine=fac.max_refine,
                                refine_mode=fac.refine_mode, refine_tol=fac.refine_tol)
        actx.fac = fac
        return beta[0]

    @staticmethod
    def backward(actx, grad_beta):
        fac = actx.fac
        v = torch.empty(fac.n_feat, dtype=torch.float64, device=fac.device)
        grad_rhs = torch.empty(fac.n_rows, dtype=torch.float64, device=fac.device)
        fl.fastlsq_backward(fac.ctx, fac.handle, grad_beta.contiguous().to(torch.float64), v,
                            grad_rhs, fac.A_op, max_iter=fac.adjoint_iters, tol=fac.adjoint_tol)
        return grad_rhs, None


class _GaussSource(torch.autograd.Function):
    @staticmethod
    def forward(actx, theta, x, ctx):
        f = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        th = theta.detach().cpu().numpy().astype(np.float64)
        fl.fastlsq_rhs(ctx, fl.GAUSS_SOURCE_2D, fl.RHS_SOURCE, th, x, 1.0, f)
        actx.ctx, actx.x, actx.th = ctx, x, th
        actx.theta_device = theta.device
        return f

    @staticmethod
    def backward(actx, grad_f):
        g = fl.fastlsq_source_grad(actx.ctx, actx.x, actx.th, grad_f.contiguous().to(torch.float64))
        return torch.as_tensor(g, dtype=torch.float64, device=actx.theta_device), None, None


class _Evaluate(torch.autograd.Function):
    @staticmethod
    def forward(actx, beta, x, W, b, scale, ctx):
        u = torch.empty(x.shape[0], dtype=torch.float64, device=x.device)
        fl.fastlsq_eval(ctx, x, W, b, scale, beta.contiguous(), u)
        actx.save = (x, W, b, scale, ctx)
        return u

    @staticmethod
    def backward(actx, g):
        x, W, b, scale, ctx = actx.save
        gb = torch.empty(W.shape[0], dtype=torch.float64, device=W.device)
        fl.fastlsq_eval_adjoint(ctx, x, W, b, scale, g.contiguous().to(torch.float64), gb)
        return gb, None, None, None, None, None


def gauss_source(ctx, theta, x):
    """s(x; theta) = sum_k a_k exp(-|x - c_k|^2 / (2 w_k^2)) at the points x (device)."""
    return _GaussSource.apply(theta, x, ctx)


def evaluate(ctx, beta, x, W, b, scale):
    """u(x) = scale * sum_j beta_j sin(W_j.x + b_j) at the points x (device)."""
    return _Evaluate.apply(beta, x, W, b, scale, ctx)

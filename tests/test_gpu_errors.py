"""Invalid arguments to the newer entry points return FASTLSQ_ERR_INVALID (raised as
FastLSQError by the binding) without launching anything, and the context stays usable."""
import numpy as np
import pytest
import torch

from paper_2602_10541_gb300 import fastlsq as fl
from paper_2602_10541_gb300 import pipeline as pl
from paper_2602_10541_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    return fl.Context(0)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _expect_invalid(fn):
    with pytest.raises(fl.FastLSQError) as e:
        fn()
    assert e.value.code == -1


def test_invalid_arguments_are_rejected(ctx):
    rng = np.random.default_rng(0)
    x, W, b = _t(rng.random((10, 2))), _t(rng.standard_normal((6, 2))), _t(rng.random(6))
    r, beta = _t(rng.standard_normal(10)), _t(rng.standard_normal(6))
    gW = torch.zeros((6, 2), dtype=torch.float64, device=DEV)
    pp_op = fl.Op(np.zeros((1, 2), np.int32), [1.0], [[1, 0]], [_t(np.ones(10))])
    # per-point terms have no place in the feature-weight gradient
    _expect_invalid(lambda: fl.fastlsq_weight_grad(ctx, x, pp_op, 1.0, W, b, 0.5, r, beta, gW))
    # contraction: a dimension beyond the limit
    _expect_invalid(lambda: ctx.check(ctx.lib.fastlsq_bandwidth_grad(ctx.handle, fl._ptr(gW), fl._ptr(W), 6, 9,
                                                                      fl._ptr(gW))))
    # residual: ld smaller than m
    _expect_invalid(lambda: ctx.check(ctx.lib.fastlsq_residual(ctx.handle, fl._ptr(gW), 4, 10, 2, fl._ptr(beta),
                                                                fl._ptr(r), fl._ptr(r))))
    # the coefficient kinds exist only for the variable-coefficient problem
    out = torch.empty(10, dtype=torch.float64, device=DEV)
    _expect_invalid(lambda: fl.fastlsq_rhs(ctx, fl.HELMHOLTZ_2D, fl.RHS_COEF, [4.0], x, 1.0, out))
    # kinds past the dimension's gradient components
    _expect_invalid(lambda: fl.fastlsq_rhs(ctx, fl.VARCOEF_2D, fl.RHS_COEF_GRAD + 2, [1.0], x, 1.0, out))
    # the 1-D kinks need a positive eps / nu
    _expect_invalid(lambda: fl.fastlsq_rhs(ctx, fl.BURGERS_1D, fl.RHS_EXACT, [0.0], x[:, :1].contiguous(), 1.0,
                                           out))
    # Newton: an unknown nonlinearity, and a continuation without stages
    w = wl.burgers1d(n_int=40, n_feat=16)
    dp = pl.upload(w, DEV)
    f = torch.zeros(w.n_int, dtype=torch.float64, device=DEV)
    g = torch.zeros(w.n_bc, dtype=torch.float64, device=DEV)
    b0 = torch.zeros(w.n_feat, dtype=torch.float64, device=DEV)
    _expect_invalid(lambda: fl.fastlsq_newton(ctx, dp.x_int, dp.x_bc, dp.op_int, 7, 1.0, w.lam_bc, f, g, dp.W,
                                              dp.b, w.scale, b0, max_iter=2))
    _expect_invalid(lambda: fl.fastlsq_newton_continuation(ctx, dp.x_int, dp.x_bc, dp.op_int, np.zeros((0, 1)),
                                                           w.nl_kind, w.nl_lam, w.lam_bc, f, g, dp.W, dp.b,
                                                           w.scale, b0))
    # the context still works
    u = torch.empty(10, dtype=torch.float64, device=DEV)
    fl.fastlsq_eval(ctx, x, W, b, 0.5, beta, u)
    assert torch.isfinite(u).all()

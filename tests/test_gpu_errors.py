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


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_waits_time_out_and_the_context_recovers(which):
    """A wait that never completes (0: an mbarrier nobody arrives on, like the
    tensor-core kernels' waits; 1: the grid barrier of the cooperative kernels with one
    CTA that never arrives) gives up after its budget (2e6 SM cycles, about a
    millisecond), raises the device flag and returns: fastlsq_sync reports
    FASTLSQ_ERR_TIMEOUT, the flag is cleared, and the context then solves correctly."""
    ctx = fl.Context(0)
    fl.fastlsq_selftest_wait(ctx, which, 2_000_000)
    with pytest.raises(fl.FastLSQError) as e:
        fl.fastlsq_sync(ctx)
    assert e.value.code == -4
    assert fl.fastlsq_sync(ctx) == 0
    # the cooperative kernels (the grid barrier) and the tensor-core kernels still work
    w = wl.helmholtz2d(n_int=1536, n_bc=256, n_feat=384)
    s = pl.LinearSolver(ctx, pl.upload(w), prec=fl.PREC_MIXED, max_refine=2)
    s.step(stats=True)
    assert s.stats.status == 0 and s.stats.tensor_core == 1
    assert pl.rel_l2(s.u_test(), s.u_exact_test()) < 1e-6
    _expect_invalid(lambda: fl.fastlsq_selftest_wait(ctx, 2, 1000))
    ctx.close()

"""GPU parity of the variable-coefficient operator (Sec. 3.8: div(nu grad u) = nu Lap u
+ grad nu . grad u, written as per-point terms of the operator) against the oracle.

- the coefficient fields of problem 10 from the GPU catalogue vs the oracle's;
- assembly of the four per-point terms, FP32 (1e-5 of the entry scale) and FP64 (1e-12),
  over several tiles with ragged edges;
- a 3-D operator with six per-point terms of orders 0..3 (the 8-term limit's use in
  d = 3), FP32 and FP64;
- solves at reduced size (FP64 1e-10 and MIXED 1e-6 of the oracle's u) and at full size
  (MIXED within 1e-6 of FP64, both near u*).
"""
import math

import numpy as np
import pytest
import torch

import oracle
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


def _entry_scale(x, alpha, coef_pt, W, scale, rw=1.0):
    """scale * rw * sum_t |c_t(x_i)| prod_k |W_jk|^alpha_tk: the entry's size without the
    trigonometric factor."""
    s = np.zeros((x.shape[0], W.shape[0]))
    for t, a in enumerate(alpha):
        m = np.prod(np.abs(W) ** np.asarray(a)[None, :], axis=1)
        s += np.abs(coef_pt[t])[:, None] * m[None, :]
    return rw * scale * s


def test_coefficient_fields_match_oracle(ctx):
    w = wl.varcoef2d(n_int=1000, n_bc=8, n_feat=8, a=0.8)
    x = _t(w.x_int)
    for kind, comp in ((fl.RHS_COEF, -1), (fl.RHS_COEF_GRAD, 0), (fl.RHS_COEF_GRAD + 1, 1)):
        out = torch.empty(w.n_int, dtype=torch.float64, device=DEV)
        fl.fastlsq_rhs(ctx, w.problem, kind, w.params, x, 1.0, out)
        np.testing.assert_allclose(out.cpu().numpy(), oracle.problem_coef(w.problem, comp, w.x_int, w.params),
                                   rtol=1e-15, atol=1e-15)
    for kind in (fl.RHS_SOURCE, fl.RHS_EXACT):
        out = torch.empty(w.n_int, dtype=torch.float64, device=DEV)
        fl.fastlsq_rhs(ctx, w.problem, kind, w.params, x, 1.0, out)
        ref = (oracle.problem_source if kind == fl.RHS_SOURCE else oracle.problem_exact)(
            w.problem, w.x_int, w.params)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("dtype", [fl.F32, fl.F64])
def test_varcoef_assembly_matches_oracle(ctx, dtype):
    w = wl.varcoef2d(n_int=301, n_bc=8, n_feat=300)
    dp = pl.upload(w, DEV, ctx=ctx)
    A = fl.colmajor(w.n_int, w.n_feat, torch.float32 if dtype == fl.F32 else torch.float64, DEV, zero=True)
    fl.fastlsq_assemble(ctx, dtype, dp.x_int, dp.op_int, 1.0, dp.W, dp.b, w.scale, A, 0)
    got = A[:, : w.n_int].double().cpu().numpy().T
    cpt = np.stack([oracle.problem_coef(w.problem, c, w.x_int, w.params) for c in (-1, -1, 0, 1)])
    alpha = [[2, 0], [0, 2], [1, 0], [0, 1]]
    ref = oracle.assemble(w.x_int, alpha, np.zeros(4), w.W, w.b, w.scale, coef_pt=cpt)
    err = np.abs(got - ref) / _entry_scale(w.x_int, alpha, cpt, w.W, w.scale)
    assert err.max() <= (1e-5 if dtype == fl.F32 else 1e-12), err.max()


@pytest.mark.parametrize("dtype", [fl.F32, fl.F64])
def test_six_per_point_terms_in_3d(ctx, dtype):
    rng = np.random.default_rng(5)
    n, nf = 260, 140
    x = rng.random((n, 3))
    W = 2.0 * rng.standard_normal((nf, 3))
    b = 2 * math.pi * rng.random(nf)
    scale = 1 / math.sqrt(nf)
    alpha = [[0, 0, 0]]
    pp_alpha = [[2, 0, 0], [0, 2, 0], [0, 0, 2], [1, 0, 0], [0, 1, 1], [1, 1, 1]]
    cpt = rng.standard_normal((6, n))
    op = fl.Op(alpha, [0.5], pp_alpha=pp_alpha, pp_coef=[_t(c) for c in cpt])
    A = fl.colmajor(n, nf, torch.float32 if dtype == fl.F32 else torch.float64, DEV, zero=True)
    fl.fastlsq_assemble(ctx, dtype, _t(x), op, 1.0, _t(W), _t(b), scale, A, 0)
    got = A[:, :n].double().cpu().numpy().T
    all_alpha = alpha + pp_alpha
    all_cpt = np.vstack([np.zeros((1, n)), cpt])
    ref = oracle.assemble(x, all_alpha, [0.5] + [0.0] * 6, W, b, scale, coef_pt=all_cpt)
    all_cpt[0] += 0.5
    err = np.abs(got - ref) / _entry_scale(x, all_alpha, all_cpt, W, scale)
    assert err.max() <= (1e-5 if dtype == fl.F32 else 1e-12), err.max()


@pytest.mark.parametrize("prec,bar", [(fl.PREC_FP64, 1e-10), (fl.PREC_MIXED, 1e-6)])
def test_varcoef_solve_matches_oracle(ctx, prec, bar):
    w = wl.varcoef2d(n_int=900, n_bc=200, n_feat=200)
    dp = pl.upload(w, DEV, ctx=ctx)
    sv = pl.LinearSolver(ctx, dp, prec=prec, max_refine=4)
    sv.build_rhs()
    sv.assemble()
    sv.solve()
    u = sv.u_test().cpu().numpy()
    cpt = np.stack([oracle.problem_coef(w.problem, c, w.x_int, w.params) for c in (-1, -1, 0, 1)])
    A = np.vstack([oracle.assemble(w.x_int, [[2, 0], [0, 2], [1, 0], [0, 1]], np.zeros(4), w.W, w.b,
                                   w.scale, coef_pt=cpt),
                   oracle.assemble(w.x_bc, [[0, 0]], [1.0], w.W, w.b, w.scale, row_weight=w.lam_bc)])
    rhs = np.concatenate([oracle.problem_source(w.problem, w.x_int, w.params),
                          w.lam_bc * oracle.problem_exact(w.problem, w.x_bc, w.params)])
    u_o = oracle.eval_u(w.x_test, w.W, w.b, w.scale, oracle.lstsq(A, rhs))
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) <= bar


def test_varcoef_full_size(ctx):
    w = wl.varcoef2d()
    dp = pl.upload(w, DEV, ctx=ctx)
    us = {}
    for prec in (fl.PREC_MIXED, fl.PREC_FP64):
        sv = pl.LinearSolver(ctx, dp, prec=prec, max_refine=2)
        sv.build_rhs()
        sv.assemble()
        sv.solve()
        us[prec] = sv.u_test().cpu().numpy()
        ue = sv.u_exact_test().cpu().numpy()
    assert np.linalg.norm(us[fl.PREC_MIXED] - us[fl.PREC_FP64]) / np.linalg.norm(us[fl.PREC_FP64]) <= 1e-6
    assert np.linalg.norm(us[fl.PREC_FP64] - ue) / np.linalg.norm(ue) <= 1e-6

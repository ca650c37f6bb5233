"""Trailing updates of the MIXED factorisation on the tcgen05 tensor cores against
the FP64 oracle and against the SIMT FP32 updates.  Two modes: the default two-level
blocking (outer blocks of 128 columns updated with K = 128, operands split into
three bf16 parts, six products, FP32 accumulation in TMEM) and the panel-by-panel
TF32x3 update (operands by TMA).

Bars: both splits keep about FP32 accuracy per product (three bf16 parts: dropped
terms below 2^-25; TF32x3: 2^-22), so R must match the oracle's Householder R to the
same 2e-5 (relative to max |R|) as the SIMT FP32 path; after refinement the
solutions meet the same bars as the SIMT path (1e-9 on nearly consistent random
systems, 1e-6 on the PDE test set).  Where the factor preconditions CGLS, the
blocked mode's R must precondition as well as the SIMT FP32 R does.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
from paper_2602_10541_gb300 import fastlsq as fl
from paper_2602_10541_gb300 import pipeline as pl
from paper_2602_10541_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = fl.Context(0)
    yield c
    fl.fastlsq_set_option(c, fl.OPT_TENSOR_CORE, 1)


def _cm(M, dtype):
    m, n = M.shape
    out = fl.colmajor(m, n, dtype, DEV, zero=True)
    out[:, :m] = torch.as_tensor(M.T, dtype=dtype, device=DEV)
    return out


def _rhs(B):
    m, k = B.shape
    out = torch.zeros((k, ((m + 3) // 4) * 4), dtype=torch.float64, device=DEV)
    out[:, :m] = torch.as_tensor(B.T, device=DEV)
    return out


def _factor_r(ctx, A, tc):
    m, n = A.shape
    fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, tc)
    _, fac, st = fl.fastlsq_lstsq(ctx, fl.PREC_MIXED, _cm(A, torch.float32), m, 0.0, None, None,
                                  A_refine=_cm(A, torch.float64), keep=True, stats=True)
    R = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    fl.fastlsq_factor_get_r(ctx, fac, R)
    fl.fastlsq_factor_destroy(ctx, fac)
    fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, 1)
    return R.cpu().numpy().T, st


# (m, n): several update tiles with ragged edges; n = 40 at m = 30000 runs the 16-wide
# panel; 300 columns leave a ragged last panel, outer block and trailing tile; 700
# columns are six outer blocks; m = 30000 with 300 columns is the blocked update over
# 16-wide inner panels, and 36864 rows is the 5-D Poisson configuration's panel height.
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("m,n", [(700, 130), (3000, 257), (1500, 300), (30000, 40), (5001, 700),
                                 (30000, 300), (36864, 160)])
def test_tensor_core_r_matches_oracle(ctx, m, n, mode):
    rng = np.random.default_rng(7 * m + n)
    A = rng.standard_normal((m, n))
    Rt, st = _factor_r(ctx, A, mode)
    assert st.tensor_core == mode
    Rs, st0 = _factor_r(ctx, A, 0)
    assert st0.tensor_core == 0
    packed, _ = oracle.qr(A)
    Ro = np.triu(packed[:n])
    scale = np.abs(Ro).max()
    assert np.abs(Rt - Ro).max() <= 2e-5 * scale
    # the two update paths differ only by FP32 rounding
    assert np.abs(Rt - Rs).max() <= 2e-5 * scale


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("m,n,mu", [(517, 77, 0.0), (2000, 130, 1e-10), (4000, 513, 0.0)])
def test_tensor_core_mixed_solve_refines_to_fp64(ctx, m, n, mu, mode):
    rng = np.random.default_rng(m + 3 * n)
    A = rng.standard_normal((m, n))
    b = A @ rng.standard_normal(n)
    B = (b + 1e-9 * np.linalg.norm(b) / np.sqrt(m) * rng.standard_normal(m))[:, None]
    ref = oracle.lstsq(A, B, mu=mu).reshape(-1)
    beta = torch.zeros((1, n), dtype=torch.float64, device=DEV)
    fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, mode)
    try:
        _, _, st = fl.fastlsq_lstsq(ctx, fl.PREC_MIXED, _cm(A, torch.float32), m, mu, _rhs(B), beta,
                                    A_refine=_cm(A, torch.float64), max_refine=4, stats=True)
    finally:
        fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, 1)
    assert st.tensor_core == mode
    np.testing.assert_allclose(beta.cpu().numpy()[0], ref, rtol=1e-9, atol=1e-9 * np.abs(ref).max())


def test_tensor_core_helmholtz_matches_oracle(ctx):
    w = wl.helmholtz2d(n_int=1536, n_bc=256, n_feat=384)
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(w.x_bc, np.zeros((1, w.d), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    f = oracle.problem_source(w.problem, w.x_int, w.params)
    g = oracle.problem_exact(w.problem, w.x_bc, w.params)
    beta_o = oracle.lstsq(np.vstack([A_int, A_bc]), np.concatenate([f, w.lam_bc * g]), mu=w.mu)
    u_orc = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta_o)
    dp = pl.upload(w)
    fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, 1)
    try:
        s = pl.LinearSolver(ctx, dp, prec=fl.PREC_MIXED, max_refine=2)
        s.step(stats=True)
    finally:
        fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, 1)
    assert s.stats.tensor_core == 1
    assert pl.rel_l2(s.u_test().cpu().numpy(), u_orc) <= 1e-6


def _inverse_operator(w):
    """FP64 operator of a Sec. 3.8 instance (-Lap rows, Dirichlet rows weighted by lam)
    with the Tikhonov rows sqrt(mu) I below, from the oracle."""
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(w.x_bc, np.zeros((1, w.d), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    return np.vstack([A_int, A_bc])


@pytest.mark.parametrize("q", [0, 1, 2])
def test_blocked_factor_preconditions_like_simt(ctx, q):
    """cond(A_mu R^{-1}) with R from the blocked tensor-core factor against R from the
    SIMT FP32 factor, on inverse-problem instances whose regularised system has a
    condition number near 1/eps32 (the systems CGLS refines): the three-part bf16
    products must not degrade the preconditioner (the TF32x3 update did: 10-170
    against 2-11).  CGLS needs about sqrt(cond) iterations, so the bar of twice the
    SIMT factor's condition number allows at most 1.41x the iterations.  The tensor
    core's own FP32 accumulation inside each MMA, which no drain schedule removes,
    keeps the blocked factor 1.2-1.6x above the SIMT one (measured 14.0-14.6 against
    8.8-11.8)."""
    w = wl.inverse_instance(q, n_int=1600, n_feat=384)
    A = _inverse_operator(w)
    m, n = A.shape
    Aug = np.vstack([A, math.sqrt(w.mu) * np.eye(n)])
    conds = {}
    for mode in (0, 1):
        fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, mode)
        try:
            _, fac, st = fl.fastlsq_lstsq(ctx, fl.PREC_MIXED, _cm(A, torch.float32), m, w.mu, None, None,
                                          A_refine=_cm(A, torch.float64), keep=True, stats=True,
                                          refine_mode=fl.REFINE_CGLS)
        finally:
            fl.fastlsq_set_option(ctx, fl.OPT_TENSOR_CORE, 1)
        assert st.tensor_core == mode
        R = torch.zeros((n, n), dtype=torch.float64, device=DEV)
        fl.fastlsq_factor_get_r(ctx, fac, R)
        fl.fastlsq_factor_destroy(ctx, fac)
        Rn = R.cpu().numpy().T
        P = scipy.linalg.solve_triangular(Rn, np.eye(n), lower=False)
        conds[mode] = np.linalg.cond(Aug @ P)
    print(f"instance {q}: cond(A R^-1) SIMT {conds[0]:.3g}, blocked tensor core {conds[1]:.3g}")
    assert conds[1] <= 2.0 * conds[0]

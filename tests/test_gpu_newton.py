"""GPU parity of Newton-Raphson (Sec. 2.4, eq. newton) against the FP64 oracle.

With a fixed number of iterations both sides take the same steps, so u on the
test set must agree (FP64 path 1e-9, MIXED 1e-6).  At full size (8192 + 1024 rows,
2048 features) the MIXED solve must agree with the FP64 GPU solve to 1e-6 and the
residual must fall by orders of magnitude in the first iterations.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_10541_gb300 import fastlsq as fl
from paper_2602_10541_gb300 import workloads as wl
from tests.golden import bratu as golden_bratu

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    return fl.Context(0)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _gpu_newton(ctx, w, prec, max_iter, tol=1e-10):
    beta = torch.zeros(w.n_feat, dtype=torch.float64, device=DEV)
    rc, st = fl.fastlsq_newton(ctx, _t(w.x_int), _t(w.x_bc), fl.Op(w.alpha, w.coef), fl.NL_EXP,
                               w.nl_lam, w.lam_bc, _t(np.zeros(w.n_int)), _t(np.zeros(w.n_bc)),
                               _t(w.W), _t(w.b), w.scale, beta, max_iter=max_iter, tol=tol,
                               mu=w.mu, prec=prec, max_refine=64, refine_tol=1e-13)
    return beta, rc, st


def _u(ctx, w, beta):
    u = torch.empty(w.x_test.shape[0], dtype=torch.float64, device=DEV)
    fl.fastlsq_eval(ctx, _t(w.x_test), _t(w.W), _t(w.b), w.scale, beta, u)
    return u.cpu().numpy()


# MIXED steps are solved by CGLS to a relative accuracy of about 2e-6 per step
# (FP32 factor as preconditioner, 64 iterations), so three steps agree to 1e-5
@pytest.mark.parametrize("prec,bar", [(fl.PREC_FP64, 1e-9), (fl.PREC_MIXED, 1e-5)])
def test_newton_steps_match_oracle(ctx, prec, bar):
    w = wl.bratu2d(n_int=1200, n_bc=256, n_feat=320)
    w.W = w.W * (2.0 / 6.0)
    iters = 3
    beta_o, st_o, it_o, hist_o = oracle.newton(w.x_int, w.x_bc, w.alpha, w.coef, oracle.NL_EXP, 1.0,
                                               w.lam_bc, np.zeros(w.n_int), np.zeros(w.n_bc), w.W,
                                               w.b, w.scale, mu=w.mu, max_iter=iters, tol=0.0)
    beta, rc, st = _gpu_newton(ctx, w, prec, iters, tol=0.0)
    assert st.iters == it_o == iters
    u_o = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta_o)
    u = _u(ctx, w, beta)
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) <= bar
    res = np.array(st.res_norm[: iters + 1])
    # the residual holds Lap u: a solution error eps shows up amplified by about
    # |W|^2 ~ sigma^2 d, so the MIXED residual history is held to 1e-4
    np.testing.assert_allclose(res[:2], hist_o[:2], rtol=1e-6 if prec == fl.PREC_FP64 else 1e-4)
    np.testing.assert_allclose(st.alpha[:iters], [1.0] * iters)


def test_newton_bratu_full_size(ctx):
    """The Bratu configuration at full size (8192 + 1024 rows, 2048 features, Newton
    from beta = 0, step test 1e-10, at most 15 iterations).  Both precisions must end on
    the step test or the iteration cap, never on a failed line search; the MIXED field
    must match the FP64 GPU field and both must match an independent finite-difference
    solution (Richardson-extrapolated 5-point scheme) on the test set."""
    w = wl.bratu2d()
    beta_m, rc_m, st_m = _gpu_newton(ctx, w, fl.PREC_MIXED, 15)
    beta_d, rc_d, st_d = _gpu_newton(ctx, w, fl.PREC_FP64, 15)
    assert rc_m in (0, 1) and rc_d in (0, 1), (rc_m, rc_d)
    assert st_m.res_norm[2] < 1e-2 * st_m.res_norm[0]
    # whether the config's step criterion (relative step <= 1e-10) was met
    print(f"bratu: MIXED status {rc_m}, {st_m.iters} iterations, last step {st_m.step_rel[st_m.iters - 1]:.2e}; "
          f"FP64 status {rc_d}, {st_d.iters} iterations, last step {st_d.step_rel[st_d.iters - 1]:.2e}")
    assert (rc_m == 0) == (st_m.step_rel[st_m.iters - 1] <= 1e-10)
    u_m, u_d = _u(ctx, w, beta_m), _u(ctx, w, beta_d)
    # the comparison is bounded by what the FP64 iteration itself still changes: 1e-6
    # plus ten times its last relative step
    bar = 1e-6 + 10 * st_d.step_rel[st_d.iters - 1]
    assert np.linalg.norm(u_m - u_d) / np.linalg.norm(u_d) <= bar
    ref = golden_bratu.bratu_reference(128)(w.x_test)
    for u in (u_m, u_d):
        err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
        print(f"bratu: rel L2 vs finite differences {err:.2e}")
        assert err <= 1e-4, err
    # the classical lambda = 1 Bratu solution peaks near 0.0784
    uc = torch.empty(1, dtype=torch.float64, device=DEV)
    fl.fastlsq_eval(ctx, _t([[0.5, 0.5]]), _t(w.W), _t(w.b), w.scale, beta_m, uc)
    assert 0.078 < uc.item() < 0.079


def _u_star(x):
    return np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) + 0.5 * x[:, 0] * x[:, 1]


def _cubic_newton(ctx, w, prec, max_iter, f, g, tol=1e-10):
    beta = torch.zeros(w.n_feat, dtype=torch.float64, device=DEV)
    rc, st = fl.fastlsq_newton(ctx, _t(w.x_int), _t(w.x_bc), fl.Op(w.alpha, w.coef), fl.NL_CUBIC,
                               w.nl_lam, w.lam_bc, f, g, _t(w.W), _t(w.b), w.scale, beta,
                               max_iter=max_iter, tol=tol, mu=w.mu, prec=prec, max_refine=64,
                               refine_tol=1e-13)
    return beta, rc, st


@pytest.mark.parametrize("name", ["nlpoisson2d", "nlhelmholtz2d"])
@pytest.mark.parametrize("prec,bar", [(fl.PREC_FP64, 1e-9), (fl.PREC_MIXED, 1e-5)])
def test_newton_cubic_steps_match_oracle(ctx, name, prec, bar):
    """The cubic Newton problems (N(u) = lam u^3, Jacobian term 3 lam u^2 H): three
    steps from beta = 0 against the oracle's, with the sources from the oracle."""
    w = getattr(wl, name)(n_int=1200, n_bc=256, n_feat=320)
    f = oracle.problem_source(w.problem, w.x_int, w.params)
    g = _u_star(w.x_bc)
    iters = 3
    beta_o, st_o, it_o, hist_o = oracle.newton(w.x_int, w.x_bc, w.alpha, w.coef, oracle.NL_CUBIC, w.nl_lam,
                                               w.lam_bc, f, g, w.W, w.b, w.scale, mu=w.mu,
                                               max_iter=iters, tol=0.0)
    beta, rc, st = _cubic_newton(ctx, w, prec, iters, _t(f), _t(g), tol=0.0)
    assert st.iters == it_o == iters
    u_o = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta_o)
    u = _u(ctx, w, beta)
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) <= bar
    np.testing.assert_allclose(st.res_norm[:2], hist_o[:2], rtol=1e-6 if prec == fl.PREC_FP64 else 1e-4)


def test_newton_nlpoisson_full_size(ctx):
    """NL-Poisson at the Bratu sizes (8192 + 1024 rows, 2048 features), sources from the
    GPU's problem catalogue: MIXED within 1e-6 of u* and of the FP64 run."""
    w = wl.nlpoisson2d()
    f = torch.empty(w.n_int, dtype=torch.float64, device=DEV)
    g = torch.empty(w.n_bc, dtype=torch.float64, device=DEV)
    fl.fastlsq_rhs(ctx, fl.NLPOISSON_2D, fl.RHS_SOURCE, w.params, _t(w.x_int), 1.0, f)
    fl.fastlsq_rhs(ctx, fl.NLPOISSON_2D, fl.RHS_EXACT, w.params, _t(w.x_bc), 1.0, g)
    np.testing.assert_allclose(g.cpu().numpy(), _u_star(w.x_bc), rtol=0, atol=1e-14)
    beta_m, rc_m, st_m = _cubic_newton(ctx, w, fl.PREC_MIXED, 12, f, g)
    beta_d, rc_d, st_d = _cubic_newton(ctx, w, fl.PREC_FP64, 12, f, g)
    u_m, u_d = _u(ctx, w, beta_m), _u(ctx, w, beta_d)
    ue = _u_star(w.x_test)
    assert np.linalg.norm(u_d - ue) / np.linalg.norm(ue) <= 1e-6
    assert np.linalg.norm(u_m - ue) / np.linalg.norm(ue) <= 1e-6
    assert np.linalg.norm(u_m - u_d) / np.linalg.norm(u_d) <= 1e-6 + 10 * st_d.step_rel[st_d.iters - 1]


# ---------------------------------------------------------------------------
# 1-D Newton problems of Sec. 3.3: Allen-Cahn (cubic, L = eps D^2 + 1) and steady
# Burgers (N = u u', whose Jacobian carries a per-point coefficient on the
# first-derivative feature), with the linear warm start and, for Burgers, the
# continuation in nu.  The oracle takes the same warm start and stages.
# ---------------------------------------------------------------------------

def _kink(name, x, c):
    s = x[:, 0] - 0.5
    return np.tanh(s / np.sqrt(2 * c)) if name == "allen_cahn1d" else -np.tanh(s / (2 * c))


def _oracle_1d(w, stages, iters):
    f = np.zeros(w.n_int)
    g = oracle.problem_exact(w.problem, w.x_bc, w.params)
    beta, *_ = oracle.newton(w.x_int, w.x_bc, w.alpha, stages[0], oracle.NL_NONE, 0.0, w.lam_bc,
                             f, g, w.W, w.b, w.scale, mu=w.mu, max_iter=1, tol=0.0)
    hists = []
    for coef in stages:
        beta, st, it, hist = oracle.newton(w.x_int, w.x_bc, w.alpha, coef, w.nl_kind, w.nl_lam,
                                           w.lam_bc, f, g, w.W, w.b, w.scale, mu=w.mu,
                                           max_iter=iters, tol=0.0, beta0=beta)
        hists.append(hist)
    return beta, hists


def _gpu_1d(ctx, w, prec, iters, stages=None):
    from paper_2602_10541_gb300 import pipeline as pl
    dp = pl.upload(w, DEV)
    f = torch.zeros(w.n_int, dtype=torch.float64, device=DEV)
    g = torch.empty(w.n_bc, dtype=torch.float64, device=DEV)
    fl.fastlsq_rhs(ctx, w.problem, fl.RHS_EXACT, w.params, dp.x_bc, 1.0, g)
    np.testing.assert_allclose(g.cpu().numpy(), _kink(w.name, w.x_bc, w.params[0]), rtol=0, atol=1e-15)
    return pl.newton_solve(ctx, dp, f, g, prec=prec, max_iter=iters, tol=0.0, stage_coef=stages)


@pytest.mark.parametrize("name", ["allen_cahn1d", "burgers1d"])
@pytest.mark.parametrize("prec,bar", [(fl.PREC_FP64, 1e-9), (fl.PREC_MIXED, 1e-5)])
def test_newton_1d_steps_match_oracle(ctx, name, prec, bar):
    """Warm start plus three Newton steps at the target eps / nu against the oracle's."""
    w = getattr(wl, name)(n_int=600, n_feat=300)
    beta_o, (hist_o,) = _oracle_1d(w, [w.coef], 3)
    beta, rc, (st,) = _gpu_1d(ctx, w, prec, 3)
    assert st.iters == 3
    u_o = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta_o)
    u = _u(ctx, w, beta)
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) <= bar
    np.testing.assert_allclose(st.res_norm[:3], hist_o[:3], rtol=1e-6 if prec == fl.PREC_FP64 else 1e-3)


@pytest.mark.parametrize("prec,bar", [(fl.PREC_FP64, 1e-8), (fl.PREC_MIXED, 1e-5)])
def test_newton_burgers_continuation_matches_oracle(ctx, prec, bar):
    """fastlsq_newton_continuation over nu = 1, 0.5, 0.2, 0.1 (three steps per stage)
    against the oracle's stage-by-stage solves."""
    w = wl.burgers1d(n_int=600, n_feat=300)
    stages = wl.burgers_stage_coef(0.1)
    beta_o, hists_o = _oracle_1d(w, list(stages), 3)
    beta, rc, sts = _gpu_1d(ctx, w, prec, 3, stages=stages)
    assert len(sts) == 4 and all(s.iters == 3 for s in sts)
    u_o = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta_o)
    u = _u(ctx, w, beta)
    assert np.linalg.norm(u - u_o) / np.linalg.norm(u_o) <= bar
    for s, h in zip(sts, hists_o):
        np.testing.assert_allclose(s.res_norm[0], h[0], rtol=1e-6 if prec == fl.PREC_FP64 else 1e-3)


@pytest.mark.parametrize("name", ["allen_cahn1d", "burgers1d"])
def test_newton_1d_full_size(ctx, name):
    """The 1-D problems at the paper's sizes (5000 interior points, 1500 features):
    MIXED and FP64 reach the exact kink to 1e-5 and agree with each other."""
    w = getattr(wl, name)()
    stages = wl.burgers_stage_coef(0.1) if name == "burgers1d" else None
    iters = 12 if stages is not None else 30
    beta_m, rc_m, st_m = _gpu_1d(ctx, w, fl.PREC_MIXED, iters, stages)
    beta_d, rc_d, st_d = _gpu_1d(ctx, w, fl.PREC_FP64, iters, stages)
    u_m, u_d = _u(ctx, w, beta_m), _u(ctx, w, beta_d)
    ue = _kink(name, w.x_test, w.params[0])
    assert np.linalg.norm(u_d - ue) / np.linalg.norm(ue) <= 1e-5
    assert np.linalg.norm(u_m - ue) / np.linalg.norm(ue) <= 1e-5
    assert np.linalg.norm(u_m - u_d) / np.linalg.norm(u_d) <= 1e-6
